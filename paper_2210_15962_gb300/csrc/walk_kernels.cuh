// Device kernels of the parallel self-avoiding-walk round (Eq. 4, Algorithm 2)
// and their launch parameters.  Shared by the plain entry points and the
// persistent batched/serving scheduler.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "walk_core.cuh"

namespace psaw {

constexpr int kWalkBlock = 128;   // threads (= walks) per block
constexpr int kTopK = 4;          // candidates kept per pass of the neighbourhood scan

// neighbourhood evaluation variants (labs_opts.kernel)
constexpr int32_t kVariantFullScan = 1;     // every Delta_j from the digit planes each step
constexpr int32_t kVariantIncremental = 2;  // stored Delta_j updated after each move
constexpr int32_t kVariantWarp = 3;         // the full scan with one warp per walk (lanes split the flips)
constexpr int32_t kVariantCta = 4;          // the full scan with one CTA per walk (its threads split the flips)

enum ErrorBits : int32_t {
  kErrRecheck = 1,   // incremental state disagreed with the XOR+popc recheck
  kErrOverflow = 2,  // a visited table ran out of slots
  kErrIncomplete = 4,  // a batch round needed for a result did not complete (a scheduling bug)
};

// search spaces: the skew-symmetric sequences of odd L, or all sequences
constexpr int32_t kSpaceSkew = 0;
constexpr int32_t kSpaceFull = 1;

// One launch = walks [g_begin, g_begin + g_count) of one round of one or more
// problems of the same L; global walk id gw = problem * walks_per_problem + walk.
struct WalkParams {
  int32_t L;
  int32_t walk_len;
  int32_t walks_per_problem;
  int32_t n_problems;
  uint32_t round;
  uint32_t g_begin;
  uint32_t g_count;
  uint32_t cap;           // visited-table slots per walk (power of two)
  int32_t kw64;           // 64-bit words per slot
  int32_t recheck_every;  // 0 = off
  const uint64_t *seeds;  // [n_problems]
  const int32_t *done;    // [n_problems], nonzero = skip (may be null)
  uint64_t *tables;       // [g_count][cap][kw64]
  // per-walk results, indexed by gw
  int32_t *w_bestE;
  int32_t *w_moves;
  int32_t *w_stuck;
  int32_t *w_best_step;
  uint32_t *w_key;        // [gw][kKeyWords]
  // per-problem accumulators
  unsigned long long *p_evals;
  unsigned long long *p_round_best;  // (E << 32) | walk, atomicMin
  // optional trajectory capture for gw in [trace_begin, trace_begin + trace_count)
  int32_t *trace_flips;   // [trace_count][walk_len]
  uint32_t trace_begin;
  uint32_t trace_count;
  int32_t *err;
  // multipliers 1, 2, 4, 2^31, 2^30 as run-time values (see Muls)
  uint32_t mul_one, mul_two, mul_four, mul_h31, mul_h30;
  // sum over walk steps of the digit planes used (for the work accounting)
  unsigned long long *plane_steps;
  int32_t variant;  // kVariantFullScan or kVariantIncremental
  int32_t space;    // kSpaceSkew or kSpaceFull
};

inline void set_muls(WalkParams &p) {
  p.mul_one = 1u;
  p.mul_two = 2u;
  p.mul_four = 4u;
  p.mul_h31 = 0x80000000u;
  p.mul_h30 = 0x40000000u;
}

struct FinalizeParams {
  int32_t n_problems;
  int32_t walks_per_problem;
  uint32_t round;
  int32_t *done;
  const uint64_t *budget;   // [n] neighbour-evaluation budget
  const int64_t *target;    // [n] target energy, < 0 = none
  const uint32_t *w_key;
  unsigned long long *p_evals;
  unsigned long long *p_round_best;
  int64_t *p_bestE;
  uint32_t *p_key;          // [n][kKeyWords]
  int32_t *p_rounds;
  int32_t *p_best_round;
  int32_t *p_best_walk;
};

// Launch one round chunk for lag-word class W (L = 2m+1 with m <= 32W).
cudaError_t launch_walk_round(int W, const WalkParams &p, cudaStream_t s);
// One round's walk kernel of lag-word class W (p.variant selects the full
// scan or the incremental kernel); defined in walk_class.cu, one object per W.
template <int W>
cudaError_t launch_walk_class(const WalkParams &p, cudaStream_t s);
extern template cudaError_t launch_walk_class<1>(const WalkParams &, cudaStream_t);
extern template cudaError_t launch_walk_class<2>(const WalkParams &, cudaStream_t);
extern template cudaError_t launch_walk_class<3>(const WalkParams &, cudaStream_t);
extern template cudaError_t launch_walk_class<4>(const WalkParams &, cudaStream_t);
extern template cudaError_t launch_walk_class<5>(const WalkParams &, cudaStream_t);
extern template cudaError_t launch_walk_class<6>(const WalkParams &, cudaStream_t);
extern template cudaError_t launch_walk_class<7>(const WalkParams &, cudaStream_t);
extern template cudaError_t launch_walk_class<8>(const WalkParams &, cudaStream_t);
cudaError_t launch_finalize(const FinalizeParams &f, cudaStream_t s);
cudaError_t launch_init_problems(int n, int64_t *p_bestE, unsigned long long *p_evals,
                                 unsigned long long *p_round_best, int32_t *done, int32_t *p_rounds,
                                 int32_t *p_best_round, int32_t *p_best_walk, uint32_t *p_key, cudaStream_t s);
// keys -> +-1 sequences: a skew key holds the D free values (Eq. 2 gives the
// rest), a full-space key the whole sequence (full = 1)
cudaError_t launch_expand(int n, int L, const uint32_t *keys, size_t key_stride, int8_t *seq_out, cudaStream_t s,
                          int full = 0);
cudaError_t launch_energy(const int8_t *seqs, int n, int L, int64_t *E_out, int32_t *err, cudaStream_t s);

inline int lag_words(int L) { return ((L - 1) / 2 + 31) / 32; }

// Visited-table slots of one walk of walk_len steps: the power of two (at
// least 64) >= factor_x10 / 10 x its walk_len + 1 pivots, plus one.  Every
// entry point sizes its tables with this one rule (factor 3 unless a batch
// is tuned otherwise: at load factor <= 1/3 a lookup reads fewer slots than
// at <= 2/3, and the walk kernel measured 2% faster at L=121 and L=223).
constexpr int kTableFactorX10 = 30;
inline uint32_t visited_table_cap(int32_t walk_len, int factor_x10 = kTableFactorX10) {
  const uint64_t need = ((uint64_t)walk_len + 1) * (uint64_t)factor_x10 / 10 + 1;
  uint64_t cap = 64;
  while (cap < need) cap <<= 1;
  return (uint32_t)cap;
}
// 32-bit words of the L - 1 lags of the full search space
inline int full_lag_words(int L) { return (L - 1 + 31) / 32; }

}  // namespace psaw
