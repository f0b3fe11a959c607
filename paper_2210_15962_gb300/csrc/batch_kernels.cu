// Persistent batch kernel: every warp repeatedly takes the next task (32
// walks of one round of one problem) from a device counter and runs it, so
// problems of different L and cost share the GPU without per-problem
// launches.  One kernel per lag-word class W (each with the register budget
// of the per-round walk kernel of that class).
#include <climits>

#include "batch.cuh"
#include "walk_device.cuh"

namespace psaw {

constexpr int kBatchMaxThreads = 256;

// Widest lag-word class whose scan runs through pattern-specialised loops: the
// classes' persistent kernels run side by side, so their code shares the SMs'
// instruction caches and is kept smaller than in the per-round kernel (with
// classes up to 4 words specialised the batched workload measured 13% slower).
constexpr int kBatchPatternMaxWords = 2;

// register budget per thread of each class: the smallest that does not spill
// (the task loop keeps more state live than the per-round kernel).  Tighter
// budgets that keep one more block resident but spill measured slower.
template <int W>
struct MaxRegsFor {
  static constexpr int value = W == 1 ? 104 : (W == 2 ? 112 : (W <= 4 ? 128 : (W == 5 ? 208 : 255)));
};

// shared memory words of one warp: mask table, then (W + 2) parked words per lane
template <int W>
constexpr int kBatchWarpWords = MaskTable<W>::kWords + (W + 2) * 32;

template <int W>
__global__ void __launch_bounds__(kBatchMaxThreads) __maxnreg__(MaxRegsFor<W>::value)
    batch_kernel(const BatchKernelParams p) {
  constexpr int T = PlanesFor<W>::value;
  constexpr int NS = W + 1;
  const int lane = threadIdx.x & 31;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t *table = p.pool + gtid * p.pool_words;
  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  // each warp's valid-lag mask table (refilled when its task's L changes) and
  // its lanes' parked best pivots
  extern __shared__ __align__(16) uint32_t batch_smem[];
  uint32_t *mask_rows = batch_smem + (size_t)(threadIdx.x >> 5) * kBatchWarpWords<W>;
  uint32_t *best_park = mask_rows + MaskTable<W>::kWords + lane;
  int rows_L = 0;
  unsigned long long planes = 0;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(p.task_next, 1u);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= p.n_tasks) break;
    const BatchTask task = p.tasks[t];
    if (p.done && p.done[task.problem]) continue;
    const BatchProblem pr = p.probs[task.problem];
    const uint32_t walk = task.chunk * 32u + (uint32_t)lane;
    const bool active = walk < (uint32_t)pr.walks;
    clear_tables_warp(table, (size_t)pr.cap * (size_t)pr.kw64, active);
    const Geometry g = make_geometry(pr.L, T);
    if (pr.L != rows_L) {  // warp-uniform: every lane took the same task
      fill_mask_rows<W>(g, mask_rows, lane, 32);
      __syncwarp();
      rows_L = pr.L;
    }
    unsigned long long packed = ~0ull;
    uint32_t evals = 0;
    WalkOut<NS> o;
    if (active) {
      run_walk<W, T, kTopK, kBatchPatternMaxWords>(g, mu, mask_rows, best_park, 32, pr.seed, walk, task.round,
                                                   pr.walk_len, table, pr.cap, pr.kw64, 0, nullptr, p.err, o);
      packed = ((unsigned long long)(uint32_t)o.bestE << 32) | walk;
      evals = (uint32_t)g.D * (uint32_t)(o.moves + o.stuck);
      planes += o.planes;
    }
    // the chunk's best (lowest E, then lowest walk) publishes its key
    unsigned long long m = packed;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xFFFFFFFFu, m, off);
      m = v < m ? v : m;
    }
    if (active && packed == m) {
      uint32_t *k = p.slot_keys + ((size_t)task.slot * p.max_chunks + task.chunk) * kKeyWords;
#pragma unroll
      for (int w = 0; w < kKeyWords; ++w) k[w] = w < NS ? o.best_key[w] : 0u;
    }
    const uint32_t ev = __reduce_add_sync(0xFFFFFFFFu, evals);
    if (lane == 0) {
      atomicMin(&p.slot_best[task.slot], m);
      atomicAdd(&p.slot_evals[task.slot], (unsigned long long)ev);
    }
  }
  if (p.plane_steps && planes) atomicAdd(p.plane_steps, planes);
}

// dynamic shared memory of a block: one mask table per warp
template <int W>
static size_t batch_smem_bytes(int block) {
  return (size_t)(block / 32) * kBatchWarpWords<W> * sizeof(uint32_t);
}

template <int W>
static cudaError_t set_batch_smem(int block) {
  return cudaFuncSetAttribute(batch_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batch_smem_bytes<W>(block));
}

template <int W>
static cudaError_t launch_batch_w(int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out) {
  int per_sm = 0;
  cudaError_t e = set_batch_smem<W>(block);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<W>, block, batch_smem_bytes<W>(block));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = per_sm * sms;
  if (grid_out) *grid_out = grid;
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  batch_kernel<W><<<grid, block, batch_smem_bytes<W>(block), s>>>(p);
  return cudaGetLastError();
}

template <int W>
static int resident_w(int block) {
  int per_sm = 0, dev = 0, sms = 0;
  if (set_batch_smem<W>(block) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<W>, block, batch_smem_bytes<W>(block)) !=
      cudaSuccess)
    return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return per_sm * sms * block;
}

cudaError_t launch_batch(int W, int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out) {
  if (block < 32 || block > kBatchMaxThreads || block % 32) return cudaErrorInvalidValue;
  switch (W) {
    case 1: return launch_batch_w<1>(block, p, s, grid_out);
    case 2: return launch_batch_w<2>(block, p, s, grid_out);
    case 3: return launch_batch_w<3>(block, p, s, grid_out);
    case 4: return launch_batch_w<4>(block, p, s, grid_out);
    case 5: return launch_batch_w<5>(block, p, s, grid_out);
    case 6: return launch_batch_w<6>(block, p, s, grid_out);
    case 7: return launch_batch_w<7>(block, p, s, grid_out);
    case 8: return launch_batch_w<8>(block, p, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

int batch_resident_lanes(int W, int block) {
  switch (W) {
    case 1: return resident_w<1>(block);
    case 2: return resident_w<2>(block);
    case 3: return resident_w<3>(block);
    case 4: return resident_w<4>(block);
    case 5: return resident_w<5>(block);
    case 6: return resident_w<6>(block);
    case 7: return resident_w<7>(block);
    case 8: return resident_w<8>(block);
    default: return 0;
  }
}

// Algorithm 1's bookkeeping for a batch launch: each problem takes its rounds
// of this launch in round order (rounds beyond its stop point, run
// speculatively, are ignored), keeping the strict best (earliest round, then
// lowest walk on ties) and stopping at the budget or the target.
__global__ void batch_finalize_kernel(const BatchFinalizeParams f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= f.n_problems || f.done[p]) return;
  for (uint32_t k = 0; k < f.n_slots[p]; ++k) {
    const uint32_t slot = f.first_slot[p] + k;
    f.evals[p] += f.slot_evals[slot];
    const unsigned long long rb = f.slot_best[slot];
    if (rb != ~0ull) {
      const int64_t E = (int64_t)(rb >> 32);
      const uint32_t w = (uint32_t)(rb & 0xFFFFFFFFu);
      if (E < f.bestE[p]) {
        f.bestE[p] = E;
        const uint32_t *src = f.slot_keys + ((size_t)slot * f.max_chunks + (w >> 5)) * kKeyWords;
        for (int i = 0; i < kKeyWords; ++i) f.key[(size_t)p * kKeyWords + i] = src[i];
        f.best_round[p] = (int32_t)f.slot_round[slot];
        f.best_walk[p] = (int32_t)w;
      }
    }
    f.rounds[p] = (int32_t)f.slot_round[slot] + 1;
    if (f.evals[p] >= f.budget[p] || (f.target[p] >= 0 && f.bestE[p] <= f.target[p])) {
      f.done[p] = 1;
      break;
    }
  }
}

cudaError_t launch_batch_finalize(const BatchFinalizeParams &f, cudaStream_t s) {
  if (f.n_problems <= 0) return cudaSuccess;
  batch_finalize_kernel<<<(f.n_problems + 127) / 128, 128, 0, s>>>(f);
  return cudaGetLastError();
}

// Reset the per-problem state of the listed slots (a serving slot taking a new request).
__global__ void init_slots_kernel(const int32_t *slots, int n, int64_t *bestE, unsigned long long *evals,
                                  int32_t *done, int32_t *rounds, int32_t *best_round, int32_t *best_walk,
                                  uint32_t *key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = slots[i];
  bestE[p] = INT64_MAX;
  evals[p] = 0;
  done[p] = 0;
  rounds[p] = 0;
  best_round[p] = -1;
  best_walk[p] = -1;
  for (int k = 0; k < kKeyWords; ++k) key[(size_t)p * kKeyWords + k] = 0u;
}

cudaError_t launch_init_slots(const int32_t *slots, int n, int64_t *bestE, unsigned long long *evals, int32_t *done,
                              int32_t *rounds, int32_t *best_round, int32_t *best_walk, uint32_t *key,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  init_slots_kernel<<<(n + 127) / 128, 128, 0, s>>>(slots, n, bestE, evals, done, rounds, best_round, best_walk, key);
  return cudaGetLastError();
}

}  // namespace psaw
