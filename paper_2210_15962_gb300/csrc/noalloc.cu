// labs_saw_round_noalloc: one round of walks whose scratch memory is a fixed
// static device array instead of memory obtained at call time.
//
// For callers that cannot allocate device memory: code whose device memory is
// owned by another allocator that must not be bypassed (a framework or a
// serving process that reserves the whole GPU up front), processes running
// under a hard device-memory quota, or code that must not perform an
// allocation on the call path.  Such a caller still provides its own input
// values and device output buffers; everything else the walks need (visited
// tables, per-walk state, counters) lives in kScratchBytes of static device
// memory that every process loading this library holds until it exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/labs.h"
#include "walk_kernels.cuh"

namespace psaw {
namespace {

constexpr size_t kScratchBytes = (size_t)LABS_NOALLOC_SCRATCH_BYTES;

// The shared scratch.  In host code this name is only a stand-in for the
// symbol, never a device address: the address is looked up per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Per-device set-up, done by the first call on each device (with that device
// current): look up the device address of the static scratch.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

__global__ void widen_kernel(int n, const int32_t *in, int64_t *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

}  // namespace
}  // namespace psaw

using namespace psaw;

extern "C" labs_status labs_saw_round_noalloc(int32_t L, uint64_t seed, uint32_t round, int32_t n_walks,
                                              int32_t walk_len, int64_t *walk_best_E, int8_t *walk_best_seq,
                                              int32_t *walk_moves, int32_t *walk_stuck, void *stream) {
  if (L < LABS_L_MIN || L > LABS_L_MAX || !(L & 1) || n_walks < 1 || walk_len < 1 || walk_len > (1 << 26) ||
      !walk_best_E || !walk_best_seq)
    return LABS_EINVAL;
  const int D = (L + 1) / 2;
  const uint32_t cap = visited_table_cap(walk_len);  // the rule labs_saw_round uses
  const int kw64 = key_words64(D);
  const size_t table_bytes = (size_t)cap * kw64 * 8;
  // layout inside the static scratch
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t o_bestE = take(sizeof(int32_t) * (size_t)n_walks);
  const size_t o_moves = take(sizeof(int32_t) * (size_t)n_walks);
  const size_t o_stuck = take(sizeof(int32_t) * (size_t)n_walks);
  const size_t o_step = take(sizeof(int32_t) * (size_t)n_walks);
  const size_t o_key = take(sizeof(uint32_t) * kKeyWords * (size_t)n_walks);
  const size_t o_evals = take(sizeof(unsigned long long));
  const size_t o_rbest = take(sizeof(unsigned long long));
  const size_t o_seed = take(sizeof(uint64_t));
  const size_t o_err = take(sizeof(int32_t));
  const size_t o_tables = take(0);
  // does not fit (compared by division: the product can exceed 64 bits)
  if (o_tables > kScratchBytes || table_bytes > (kScratchBytes - o_tables) / (size_t)n_walks) return LABS_ENOMEM;

  cudaStream_t s = (cudaStream_t)stream;
  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return LABS_ECUDA;
  char *b = (char *)base;

  WalkParams p{};
  p.L = L;
  p.walk_len = walk_len;
  p.walks_per_problem = n_walks;
  p.n_problems = 1;
  p.round = round;
  p.g_begin = 0;
  p.g_count = (uint32_t)n_walks;
  p.cap = cap;
  p.kw64 = kw64;
  p.recheck_every = 0;
  p.seeds = (const uint64_t *)(b + o_seed);
  p.done = nullptr;
  p.tables = (uint64_t *)(b + o_tables);  // zeroed by the walk kernel itself
  p.w_bestE = (int32_t *)(b + o_bestE);
  p.w_moves = (int32_t *)(b + o_moves);
  p.w_stuck = (int32_t *)(b + o_stuck);
  p.w_best_step = (int32_t *)(b + o_step);
  p.w_key = (uint32_t *)(b + o_key);
  p.p_evals = (unsigned long long *)(b + o_evals);
  p.p_round_best = (unsigned long long *)(b + o_rbest);
  p.err = (int32_t *)(b + o_err);
  p.trace_flips = nullptr;
  p.trace_begin = 0;
  p.trace_count = 0;
  p.plane_steps = nullptr;
  p.variant = kVariantFullScan;
  set_muls(p);

  // counters and the error word start at zero (the scratch keeps the previous
  // call's contents); the seed is the round's only input value
  e = cudaMemsetAsync(b + o_evals, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + o_rbest, 0xFF, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + o_err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_seed, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_walk_round(lag_words(L), p, s);
  if (e == cudaSuccess) e = launch_expand(n_walks, L, p.w_key, kKeyWords, walk_best_seq, s);
  if (e == cudaSuccess) {
    widen_kernel<<<(n_walks + 255) / 256, 256, 0, s>>>(n_walks, p.w_bestE, walk_best_E);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && walk_moves)
    e = cudaMemcpyAsync(walk_moves, p.w_moves, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && walk_stuck)
    e = cudaMemcpyAsync(walk_stuck, p.w_stuck, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToDevice, s);
  int32_t err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, b + o_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LABS_ECUDA;
  if (err & kErrOverflow) return LABS_EOVERFLOW;
  return LABS_OK;
}
