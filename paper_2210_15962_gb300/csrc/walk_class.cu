// The walk kernels of one lag-word class W (Eq. 4 and Algorithm 2 of arXiv
// 2210.15962): the full-scan kernel, the incremental variant and the kernel
// of the full search space (all length-L sequences).  This file is
// compiled once per class with -DPSAW_W=W (1..8), so that the classes' large,
// pattern-specialised kernels build in parallel.
#include "walk_cta.cuh"
#include "walk_device.cuh"
#include "walk_warp.cuh"

#ifndef PSAW_W
#error "walk_class.cu is compiled once per lag-word class with -DPSAW_W=1..8"
#endif

namespace psaw {

// Widest lag-word class whose scan runs through loops specialised for the
// pattern of active word sides.  Wider classes measured slower with
// specialised runs than with one loop that keeps every word two-sided: four
// words 9% at L=223 and 40% at L=255 (with the flip loop unrolled twice and 4
// blocks per SM, 24% and 68% faster than the specialised runs with 3 blocks),
// five to eight words 1.3-2.4x.
constexpr int kWalkPatternMaxWords = 3;

// One thread = one walk (Algorithm 2 with one lane in place of one block).
// The warp zeroes the visited tables of its live lanes, then every lane runs
// its walk (run_walk) and publishes its best to the round's accumulators.
template <int W, int T, int K, int MINB>
__global__ void __launch_bounds__(kWalkBlock, MINB) walk_kernel(const WalkParams p) {
  constexpr int NS = W + 1;
  const uint32_t lid = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t table_words = (size_t)p.cap * (size_t)p.kw64;
  const uint32_t gw = p.g_begin + lid;
  const uint32_t prob = gw / (uint32_t)p.walks_per_problem;
  const uint32_t walk = gw - prob * (uint32_t)p.walks_per_problem;
  const bool live = lid < p.g_count && !(p.done && p.done[prob]);
  uint64_t *table = p.tables + (size_t)lid * table_words;
  const Geometry g = make_geometry(p.L, T);
  __shared__ __align__(16) uint32_t mask_rows[MaskTable<W>::kWords];
  __shared__ uint32_t best_park[(NS + 1) * kWalkBlock];
  fill_mask_rows<W>(g, mask_rows, threadIdx.x, blockDim.x);
  __syncthreads();
  clear_tables_warp(table, table_words, live);
  if (!live) return;

  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  int32_t *trace = nullptr;
  if (p.trace_flips && gw - p.trace_begin < p.trace_count)
    trace = p.trace_flips + (size_t)(gw - p.trace_begin) * (size_t)p.walk_len;
  WalkOut<NS> o;
  run_walk<W, T, K, kWalkPatternMaxWords, ScanUnroll<W>::value>(g, mu, mask_rows, best_park + threadIdx.x, kWalkBlock,
                                                                p.seeds[prob], walk, p.round, p.walk_len, table, p.cap,
                                                                p.kw64, p.recheck_every, trace, p.err, o);
  p.w_bestE[gw] = o.bestE;
  p.w_moves[gw] = o.moves;
  p.w_stuck[gw] = o.stuck;
  p.w_best_step[gw] = o.best_step;
#pragma unroll
  for (int w = 0; w < kKeyWords; ++w) p.w_key[(size_t)gw * kKeyWords + w] = w < NS ? o.best_key[w] : 0u;
  atomicAdd(&p.p_evals[prob], (unsigned long long)g.D * (unsigned long long)(o.moves + o.stuck));
  if (p.plane_steps) atomicAdd(p.plane_steps, o.planes);
  atomicMin(&p.p_round_best[prob], ((unsigned long long)(uint32_t)o.bestE << 32) | walk);
}

// The incremental variant: same contract as walk_kernel; each lane keeps its
// correlations and neighbour deltas in dynamic shared memory, lane-major.
template <int W, int K, int MINB>
__global__ void __launch_bounds__(kWalkBlock, MINB) walk_kernel_incr(const WalkParams p) {
  constexpr int NS = W + 1;
  using CT = typename IncrTypes<W>::CT;
  using DT = typename IncrTypes<W>::DT;
  extern __shared__ __align__(16) unsigned char incr_smem[];
  const uint32_t lid = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t table_words = (size_t)p.cap * (size_t)p.kw64;
  const uint32_t gw = p.g_begin + lid;
  const uint32_t prob = gw / (uint32_t)p.walks_per_problem;
  const uint32_t walk = gw - prob * (uint32_t)p.walks_per_problem;
  const bool live = lid < p.g_count && !(p.done && p.done[prob]);
  uint64_t *table = p.tables + (size_t)lid * table_words;
  clear_tables_warp(table, table_words, live);
  if (!live) return;
  const Geometry g = make_geometry(p.L, PlanesFor<W>::value);
  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  CT *Cs = reinterpret_cast<CT *>(incr_smem);
  DT *Ds = reinterpret_cast<DT *>(incr_smem + (size_t)g.m * blockDim.x * sizeof(CT) + 15) ;
  Ds = reinterpret_cast<DT *>((reinterpret_cast<uintptr_t>(Ds)) & ~(uintptr_t)15);
  const IncrView<CT, DT> v{Cs + threadIdx.x, Ds + threadIdx.x, (int)blockDim.x};
  int32_t *trace = nullptr;
  if (p.trace_flips && gw - p.trace_begin < p.trace_count)
    trace = p.trace_flips + (size_t)(gw - p.trace_begin) * (size_t)p.walk_len;
  WalkOut<NS> o;
  run_walk_incr<W, CT, DT, K>(g, mu, v, p.seeds[prob], walk, p.round, p.walk_len, table, p.cap, p.kw64,
                              p.recheck_every, trace, p.err, o);
  p.w_bestE[gw] = o.bestE;
  p.w_moves[gw] = o.moves;
  p.w_stuck[gw] = o.stuck;
  p.w_best_step[gw] = o.best_step;
#pragma unroll
  for (int w = 0; w < kKeyWords; ++w) p.w_key[(size_t)gw * kKeyWords + w] = w < NS ? o.best_key[w] : 0u;
  atomicAdd(&p.p_evals[prob], (unsigned long long)g.D * (unsigned long long)(o.moves + o.stuck));
  atomicMin(&p.p_round_best[prob], ((unsigned long long)(uint32_t)o.bestE << 32) | walk);
}

// resident blocks the incremental variant of each class is compiled for
template <int W>
struct MinBlocksIncr {
  static constexpr int value = W == 1 ? 8 : (W == 2 ? 8 : (W <= 4 ? 5 : 3));
};

template <int W>
static size_t incr_smem_bytes(int L, int block) {
  using CT = typename IncrTypes<W>::CT;
  using DT = typename IncrTypes<W>::DT;
  const int m = (L - 1) / 2, D = (L + 1) / 2;
  return ((size_t)m * block * sizeof(CT) + 15) / 16 * 16 + (size_t)D * block * sizeof(DT);
}

template <int W>
static cudaError_t launch_w_incr(const WalkParams &p, cudaStream_t s) {
  const unsigned blocks = (p.g_count + kWalkBlock - 1) / kWalkBlock;
  const size_t smem = incr_smem_bytes<W>(p.L, kWalkBlock);
  auto kern = walk_kernel_incr<W, kTopK, MinBlocksIncr<W>::value>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kWalkBlock, smem, s>>>(p);
  return cudaGetLastError();
}

template <int W>
static cudaError_t launch_w(const WalkParams &p, cudaStream_t s) {
  constexpr int T = PlanesFor<W>::value;
  const unsigned blocks = (p.g_count + kWalkBlock - 1) / kWalkBlock;
  walk_kernel<W, T, kTopK, MinBlocksFor<W>::value><<<blocks, kWalkBlock, 0, s>>>(p);
  return cudaGetLastError();
}

// One warp = one walk (walk_warp.cuh): same contract as walk_kernel; the
// block's warps run walks lid = 4 * block + warp, each lane a share of its
// walk's flips.
template <int W, int T, int K, int MINB>
__global__ void __launch_bounds__(kWalkBlock, MINB) walk_kernel_warp(const WalkParams p) {
  constexpr int NS = W + 1;
  constexpr int kWarps = kWalkBlock / 32;
  constexpr int kSm = WarpWalkSmem<W>::kWords;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lid = blockIdx.x * kWarps + warp;
  const size_t table_words = (size_t)p.cap * (size_t)p.kw64;
  const uint32_t gw = p.g_begin + lid;
  const uint32_t prob = gw / (uint32_t)p.walks_per_problem;
  const uint32_t walk = gw - prob * (uint32_t)p.walks_per_problem;
  const bool live = lid < p.g_count && !(p.done && p.done[prob]);  // the same on the whole warp
  uint64_t *table = p.tables + (size_t)lid * table_words;
  const Geometry g = make_geometry(p.L, T);
  __shared__ __align__(16) uint32_t mask_rows[MaskTable<W>::kWords];
  __shared__ uint32_t warp_sm[kWarps * kSm];
  fill_mask_rows<W>(g, mask_rows, threadIdx.x, blockDim.x);
  __syncthreads();
  if (!live) return;
  // the walk's table, zeroed by the warp with 16-byte stores (table_words is even)
  uint4 *t4 = reinterpret_cast<uint4 *>(table);
  for (size_t i = (size_t)lane; i < table_words / 2; i += 32) t4[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  int32_t *trace = nullptr;
  if (p.trace_flips && gw - p.trace_begin < p.trace_count)
    trace = p.trace_flips + (size_t)(gw - p.trace_begin) * (size_t)p.walk_len;
  WalkOut<NS> o;
  run_walk_warp<W, T, K>(g, mu, mask_rows, warp_sm + warp * kSm, p.seeds[prob], walk, p.round, p.walk_len, table,
                         p.cap, p.kw64, p.recheck_every, trace, p.err, o);
  if (lane != 0) return;
  p.w_bestE[gw] = o.bestE;
  p.w_moves[gw] = o.moves;
  p.w_stuck[gw] = o.stuck;
  p.w_best_step[gw] = o.best_step;
#pragma unroll
  for (int w = 0; w < kKeyWords; ++w) p.w_key[(size_t)gw * kKeyWords + w] = w < NS ? o.best_key[w] : 0u;
  atomicAdd(&p.p_evals[prob], (unsigned long long)g.D * (unsigned long long)(o.moves + o.stuck));
  if (p.plane_steps) atomicAdd(p.plane_steps, (unsigned long long)o.planes);
  atomicMin(&p.p_round_best[prob], ((unsigned long long)(uint32_t)o.bestE << 32) | walk);
}

// resident blocks the warp variant is compiled for: 6 at two words (7
// spilled); one more than the full-space kernel at three and five to eight
// words (8192 walks of 2048 steps: +3% at L=161, +4% at L=301, +7% at 383,
// +14% at 449, +10% at 511); four words spill with 5
template <int W>
struct MinBlocksWarp {
  static constexpr int value = W == 1 ? 8 : (W == 2 ? 6 : (W == 3 ? 5 : (W <= 6 ? 4 : 3)));
};

template <int W>
static cudaError_t launch_w_warp(const WalkParams &p, cudaStream_t s) {
  constexpr int T = PlanesFor<W>::value;
  const unsigned blocks = (p.g_count + kWalkBlock / 32 - 1) / (kWalkBlock / 32);
  walk_kernel_warp<W, T, kTopK, MinBlocksWarp<W>::value><<<blocks, kWalkBlock, 0, s>>>(p);
  return cudaGetLastError();
}

// One CTA = one walk (walk_cta.cuh): same contract as walk_kernel; block b
// runs walk lid = b, its kWalkBlock threads splitting the walk's flips.
template <int W, int T, int K, int MINB>
__global__ void __launch_bounds__(kWalkBlock, MINB) walk_kernel_cta(const WalkParams p) {
  constexpr int NS = W + 1;
  const uint32_t lid = blockIdx.x;
  const size_t table_words = (size_t)p.cap * (size_t)p.kw64;
  const uint32_t gw = p.g_begin + lid;
  const uint32_t prob = gw / (uint32_t)p.walks_per_problem;
  const uint32_t walk = gw - prob * (uint32_t)p.walks_per_problem;
  const bool live = lid < p.g_count && !(p.done && p.done[prob]);  // the same on every thread of the block
  uint64_t *table = p.tables + (size_t)lid * table_words;
  const Geometry g = make_geometry(p.L, T);
  __shared__ __align__(16) uint32_t mask_rows[MaskTable<W>::kWords];
  __shared__ uint32_t cta_sm[CtaWalkSmem<W>::kWords];
  fill_mask_rows<W>(g, mask_rows, threadIdx.x, blockDim.x);
  if (!live) return;
  // the walk's table, zeroed by the block with 16-byte stores (table_words is even)
  uint4 *t4 = reinterpret_cast<uint4 *>(table);
  for (size_t i = threadIdx.x; i < table_words / 2; i += blockDim.x) t4[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();  // the mask table and the zeroed table are visible to the block
  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  int32_t *trace = nullptr;
  if (p.trace_flips && gw - p.trace_begin < p.trace_count)
    trace = p.trace_flips + (size_t)(gw - p.trace_begin) * (size_t)p.walk_len;
  WalkOut<NS> o;
  run_walk_cta<W, T, K>(g, mu, mask_rows, cta_sm, p.seeds[prob], walk, p.round, p.walk_len, table, p.cap, p.kw64,
                        p.recheck_every, trace, p.err, o);
  if (threadIdx.x != 0) return;
  p.w_bestE[gw] = o.bestE;
  p.w_moves[gw] = o.moves;
  p.w_stuck[gw] = o.stuck;
  p.w_best_step[gw] = o.best_step;
#pragma unroll
  for (int w = 0; w < kKeyWords; ++w) p.w_key[(size_t)gw * kKeyWords + w] = w < NS ? o.best_key[w] : 0u;
  atomicAdd(&p.p_evals[prob], (unsigned long long)g.D * (unsigned long long)(o.moves + o.stuck));
  if (p.plane_steps) atomicAdd(p.plane_steps, (unsigned long long)o.planes);
  atomicMin(&p.p_round_best[prob], ((unsigned long long)(uint32_t)o.bestE << 32) | walk);
}

template <int W>
static cudaError_t launch_w_cta(const WalkParams &p, cudaStream_t s) {
  constexpr int T = PlanesFor<W>::value;
  walk_kernel_cta<W, T, kTopK, MinBlocksWarp<W>::value><<<p.g_count, kWalkBlock, 0, s>>>(p);
  return cudaGetLastError();
}

// The full search space (full_core.cuh): same contract as walk_kernel with L
// flips per step and the whole sequence as key (kKeyWords >= W + 1 words).
template <int W, int T, int K, int MINB>
__global__ void __launch_bounds__(kWalkBlock, MINB) full_walk_kernel(const WalkParams p) {
  constexpr int NS = W + 1;
  const uint32_t lid = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t table_words = (size_t)p.cap * (size_t)p.kw64;
  const uint32_t gw = p.g_begin + lid;
  const uint32_t prob = gw / (uint32_t)p.walks_per_problem;
  const uint32_t walk = gw - prob * (uint32_t)p.walks_per_problem;
  const bool live = lid < p.g_count && !(p.done && p.done[prob]);
  uint64_t *table = p.tables + (size_t)lid * table_words;
  __shared__ __align__(16) uint32_t mask_rows[FullMaskTable<W>::kWords];
  fill_full_mask_rows<W>(p.L, mask_rows, threadIdx.x, blockDim.x);
  __syncthreads();
  clear_tables_warp(table, table_words, live);
  if (!live) return;

  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  int32_t *trace = nullptr;
  if (p.trace_flips && gw - p.trace_begin < p.trace_count)
    trace = p.trace_flips + (size_t)(gw - p.trace_begin) * (size_t)p.walk_len;
  WalkOut<NS> o;
  run_walk_full<W, T, K>(p.L, mu, mask_rows, p.seeds[prob], walk, p.round, p.walk_len, table, p.cap, p.kw64,
                         p.recheck_every, trace, p.err, o);
  p.w_bestE[gw] = o.bestE;
  p.w_moves[gw] = o.moves;
  p.w_stuck[gw] = o.stuck;
  p.w_best_step[gw] = o.best_step;
#pragma unroll
  for (int w = 0; w < kKeyWords; ++w) p.w_key[(size_t)gw * kKeyWords + w] = w < NS ? o.best_key[w] : 0u;
  atomicAdd(&p.p_evals[prob], (unsigned long long)p.L * (unsigned long long)(o.moves + o.stuck));
  if (p.plane_steps) atomicAdd(p.plane_steps, o.planes);
  atomicMin(&p.p_round_best[prob], ((unsigned long long)(uint32_t)o.bestE << 32) | walk);
}

template <int W>
static cudaError_t launch_full(const WalkParams &p, cudaStream_t s) {
  constexpr int T = FullPlanesFor<W>::value;
  const unsigned blocks = (p.g_count + kWalkBlock - 1) / kWalkBlock;
  full_walk_kernel<W, T, kTopK, MinBlocksFull<W>::value><<<blocks, kWalkBlock, 0, s>>>(p);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_walk_class(const WalkParams &p, cudaStream_t s) {
  if (p.space == kSpaceFull) return launch_full<W>(p, s);
  if (p.variant == kVariantIncremental) return launch_w_incr<W>(p, s);
  if (p.variant == kVariantWarp) return launch_w_warp<W>(p, s);
  if (p.variant == kVariantCta) return launch_w_cta<W>(p, s);
  return launch_w<W>(p, s);
}

template cudaError_t launch_walk_class<PSAW_W>(const WalkParams &p, cudaStream_t s);

}  // namespace psaw
