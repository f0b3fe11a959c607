// Kernels of one round of parallel contiguous self-avoiding walks (Eq. 4 and
// Algorithm 2 of arXiv 2210.15962), the per-round best reduction of
// Algorithm 1, the key -> sequence expansion (Eq. 2) and the Eq. 1 energy.
#include <climits>

#include "walk_device.cuh"

namespace psaw {

// Widest lag-word class whose scan runs through pattern-specialised loops.
constexpr int kWalkPatternMaxWords = 4;

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
  run_walk<W, T, K, kWalkPatternMaxWords>(g, mu, mask_rows, best_park + threadIdx.x, kWalkBlock, p.seeds[prob], walk, p.round, p.walk_len,
                    table, p.cap, p.kw64, p.recheck_every, trace, p.err, o);
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

cudaError_t launch_walk_round(int W, const WalkParams &p, cudaStream_t s) {
  if (p.g_count == 0) return cudaSuccess;
  if (p.variant == kVariantIncremental) {
    switch (W) {
      case 1: return launch_w_incr<1>(p, s);
      case 2: return launch_w_incr<2>(p, s);
      case 3: return launch_w_incr<3>(p, s);
      case 4: return launch_w_incr<4>(p, s);
      case 5: return launch_w_incr<5>(p, s);
      case 6: return launch_w_incr<6>(p, s);
      case 7: return launch_w_incr<7>(p, s);
      case 8: return launch_w_incr<8>(p, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (W) {
    case 1: return launch_w<1>(p, s);
    case 2: return launch_w<2>(p, s);
    case 3: return launch_w<3>(p, s);
    case 4: return launch_w<4>(p, s);
    case 5: return launch_w<5>(p, s);
    case 6: return launch_w<6>(p, s);
    case 7: return launch_w<7>(p, s);
    case 8: return launch_w<8>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

// Algorithm 1's per-round bookkeeping, one thread per problem: a round best
// strictly below the running best replaces it (so the earliest round wins
// ties, and inside a round the lowest walk index wins through the atomicMin
// key); then the budget / target stop rule is applied.
__global__ void finalize_kernel(const FinalizeParams f) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= f.n_problems || f.done[p]) return;
  const unsigned long long rb = f.p_round_best[p];
  f.p_round_best[p] = ~0ull;
  if (rb != ~0ull) {
    const int64_t E = (int64_t)(rb >> 32);
    const uint32_t w = (uint32_t)(rb & 0xFFFFFFFFu);
    if (E < f.p_bestE[p]) {
      f.p_bestE[p] = E;
      const size_t gw = (size_t)p * (size_t)f.walks_per_problem + w;
      for (int i = 0; i < kKeyWords; ++i) f.p_key[(size_t)p * kKeyWords + i] = f.w_key[gw * kKeyWords + i];
      f.p_best_round[p] = (int32_t)f.round;
      f.p_best_walk[p] = (int32_t)w;
    }
  }
  f.p_rounds[p] = (int32_t)f.round + 1;
  if (f.p_evals[p] >= f.budget[p] || (f.target[p] >= 0 && f.p_bestE[p] <= f.target[p])) f.done[p] = 1;
}

cudaError_t launch_finalize(const FinalizeParams &f, cudaStream_t s) {
  finalize_kernel<<<(f.n_problems + 127) / 128, 128, 0, s>>>(f);
  return cudaGetLastError();
}

__global__ void init_problems_kernel(int n, int64_t *p_bestE, unsigned long long *p_evals,
                                     unsigned long long *p_round_best, int32_t *done, int32_t *p_rounds,
                                     int32_t *p_best_round, int32_t *p_best_walk, uint32_t *p_key) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  p_bestE[p] = INT64_MAX;
  p_evals[p] = 0;
  p_round_best[p] = ~0ull;
  done[p] = 0;
  p_rounds[p] = 0;
  p_best_round[p] = -1;
  p_best_walk[p] = -1;
  for (int i = 0; i < kKeyWords; ++i) p_key[(size_t)p * kKeyWords + i] = 0u;
}

cudaError_t launch_init_problems(int n, int64_t *p_bestE, unsigned long long *p_evals,
                                 unsigned long long *p_round_best, int32_t *done, int32_t *p_rounds,
                                 int32_t *p_best_round, int32_t *p_best_walk, uint32_t *p_key, cudaStream_t s) {
  init_problems_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, p_bestE, p_evals, p_round_best, done, p_rounds,
                                                      p_best_round, p_best_walk, p_key);
  return cudaGetLastError();
}

// Eq. 2: sequence s_0..s_{L-1} (+1/-1) from the D key bits (bit 1 <-> -1).
__global__ void expand_kernel(int n, int L, const uint32_t *keys, size_t key_stride, int8_t *seq_out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * (size_t)L) return;
  const int p = (int)(idx / (size_t)L);
  const int a = (int)(idx - (size_t)p * (size_t)L);
  const int c = (L - 1) / 2;
  const uint32_t *k = keys + (size_t)p * key_stride;
  uint32_t b;
  if (a <= c) {
    b = (k[a >> 5] >> (a & 31)) & 1u;
  } else {
    const int i = a - c, src = c - i;
    b = ((k[src >> 5] >> (src & 31)) & 1u) ^ (uint32_t)(i & 1);
  }
  seq_out[(size_t)p * L + a] = b ? (int8_t)-1 : (int8_t)1;
}

cudaError_t launch_expand(int n, int L, const uint32_t *keys, size_t key_stride, int8_t *seq_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t total = (size_t)n * (size_t)L;
  expand_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, L, keys, key_stride, seq_out);
  return cudaGetLastError();
}

// Eq. 1 for arbitrary +-1 sequences: one warp per sequence, the sequence
// bit-packed in shared memory, lanes split the lags, each C_k by XOR + popc
// of the sequence against itself shifted by k.
constexpr int kEnergyWarps = 4;

__global__ void energy_kernel(const int8_t *seqs, int n, int L, int64_t *E_out, int32_t *err) {
  extern __shared__ uint32_t sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seq = blockIdx.x * kEnergyWarps + warp;
  const int NW = (L + 31) / 32;
  uint32_t *bits = sm + (size_t)warp * (NW + 1);
  if (seq < n) {
    const int8_t *s = seqs + (size_t)seq * L;
    for (int w = lane; w <= NW; w += 32) {
      uint32_t v = 0;
      if (w < NW) {
        for (int b = 0; b < 32; ++b) {
          const int pos = 32 * w + b;
          if (pos < L) {
            const int8_t x = s[pos];
            if (x != 1 && x != -1) atomicOr(err, 1);
            v |= (x < 0 ? 1u : 0u) << b;
          }
        }
      }
      bits[w] = v;
    }
  }
  __syncwarp();
  if (seq >= n) return;
  long long acc = 0;
  for (int k = 1 + lane; k < L; k += 32) {
    const int pairs = L - k;
    const int ws = k >> 5;
    const uint32_t bs = (uint32_t)(k & 31);
    int dis = 0;
    for (int w = 0; 32 * w < pairs; ++w) {
      const uint32_t lo = bits[w + ws];
      const uint32_t hi = (w + ws + 1 <= NW) ? bits[w + ws + 1] : 0u;
      const uint32_t sh = fshr(lo, hi, bs);
      dis += (int)popc32((bits[w] ^ sh) & low_mask_word(pairs, w));
    }
    const long long C = pairs - 2 * dis;
    acc += C * C;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if (lane == 0) E_out[seq] = acc;
}

cudaError_t launch_energy(const int8_t *seqs, int n, int L, int64_t *E_out, int32_t *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int NW = (L + 31) / 32;
  const size_t smem = (size_t)kEnergyWarps * (NW + 1) * sizeof(uint32_t);
  energy_kernel<<<(n + kEnergyWarps - 1) / kEnergyWarps, 32 * kEnergyWarps, smem, s>>>(seqs, n, L, E_out, err);
  return cudaGetLastError();
}

}  // namespace psaw
