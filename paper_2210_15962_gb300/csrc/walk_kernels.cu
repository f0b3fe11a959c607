// Kernels of one round of parallel contiguous self-avoiding walks (Eq. 4 and
// Algorithm 2 of arXiv 2210.15962): the dispatch to the per-class walk
// kernels (walk_class.cu), the per-round best reduction of Algorithm 1, the
// key -> sequence expansion (Eq. 2) and the Eq. 1 energy.
#include <climits>

#include "walk_device.cuh"

namespace psaw {

cudaError_t launch_walk_round(int W, const WalkParams &p, cudaStream_t s) {
  if (p.g_count == 0) return cudaSuccess;
  switch (W) {
    case 1: return launch_walk_class<1>(p, s);
    case 2: return launch_walk_class<2>(p, s);
    case 3: return launch_walk_class<3>(p, s);
    case 4: return launch_walk_class<4>(p, s);
    case 5: return launch_walk_class<5>(p, s);
    case 6: return launch_walk_class<6>(p, s);
    case 7: return launch_walk_class<7>(p, s);
    case 8: return launch_walk_class<8>(p, s);
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
__global__ void expand_kernel(int n, int L, const uint32_t *keys, size_t key_stride, int8_t *seq_out, int full) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * (size_t)L) return;
  const int p = (int)(idx / (size_t)L);
  const int a = (int)(idx - (size_t)p * (size_t)L);
  const uint32_t b = sequence_bit(keys + (size_t)p * key_stride, L, a, full != 0);
  seq_out[(size_t)p * L + a] = b ? (int8_t)-1 : (int8_t)1;
}

cudaError_t launch_expand(int n, int L, const uint32_t *keys, size_t key_stride, int8_t *seq_out, cudaStream_t s,
                          int full) {
  if (n <= 0) return cudaSuccess;
  const size_t total = (size_t)n * (size_t)L;
  expand_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, L, keys, key_stride, seq_out, full);
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
