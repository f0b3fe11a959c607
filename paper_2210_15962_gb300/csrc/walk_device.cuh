// Device-side body of one contiguous self-avoiding walk (Eq. 3, Algorithm 2)
// on one lane, shared by the per-round walk kernel and the persistent batch
// kernel, plus small warp helpers.
#pragma once
#include <type_traits>
#include "full_core.cuh"
#include "walk_incr.cuh"
#include "walk_kernels.cuh"

namespace psaw {

// digit planes used for lag-word class W (covers every L with m <= 32W)
template <int W>
struct PlanesFor {
  static constexpr int value = W == 1 ? 6 : (W == 2 ? 7 : (W <= 4 ? 8 : 9));
};

// resident blocks of kWalkBlock walks per SM each class of the one-walk-per-
// lane kernel is compiled for (the register budget per thread is
// 65536 / (128 * MINB)); seven and eight words measured 8% and 4% faster with
// 3 blocks (168 registers) than with 2, while 5 blocks at three words and 4 at
// five lost 7% and 4%
template <int W>
struct MinBlocksFor {
  static constexpr int value = W == 1 ? 8 : (W == 2 ? 7 : (W <= 4 ? 4 : 3));
};

// The same for the full-space kernel (full_core.cuh), whose scan keeps more
// state per word: 3 blocks at seven words (+2% at L=200), 2 at eight (3
// spill there).
template <int W>
struct MinBlocksFull {
  static constexpr int value = W == 1 ? 8 : (W == 2 ? 7 : (W <= 4 ? 4 : (W <= 7 ? 3 : 2)));
};

// Flips of the scan's loop unrolled per iteration in the one-walk-per-lane
// kernel: two at four to seven words (independent popcount chains for the
// few resident warps: +3% at L=223, +4%, +3% and +2% at L=301, 383, 449),
// one elsewhere (two lost 1.5% at two words, 30% at three, and 1% at
// eight; at three words, the widest class with pattern-specialised scan
// loops, the unrolled code no longer fits the instruction caches: the same
// instructions and registers, four times the instruction-fetch stalls)
template <int W>
struct ScanUnroll {
  static constexpr int value = (W >= 4 && W <= 7) ? 2 : 1;
};

template <int NS>
struct WalkOut {
  int32_t bestE, best_step, moves, stuck;
  uint32_t best_key[NS];
  unsigned long long planes;  // sum over steps of the digit planes scanned
};

// Zero the `words` 64-bit words of every live lane's table with coalesced
// 16-byte stores by the whole warp.  All 32 lanes must call it.
__device__ __forceinline__ void clear_tables_warp(uint64_t *my_table, size_t words, bool live) {
  const int lane = threadIdx.x & 31;
  const uint32_t live_lanes = __ballot_sync(0xFFFFFFFFu, live);
  const size_t n16 = words / 2;
  for (int l = 0; l < 32; ++l) {
    const unsigned long long base = __shfl_sync(0xFFFFFFFFu, (unsigned long long)my_table, l);
    if ((live_lanes >> l) & 1u) {
      uint4 *b = reinterpret_cast<uint4 *>(base);
      for (size_t i = (size_t)lane; i < n16; i += 32) b[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  __syncwarp();
}

// One walk: random P_1, then walk_len steps of "evaluate all D flips -> best
// unvisited neighbour (ties to the lowest flip) -> insert -> update C, E ->
// keep the strict best".  The scan keeps the K smallest (Delta, flip) keys; if
// all are visited it rescans above the last one, so the choice is exactly the
// minimum over unvisited neighbours.  `table` must be zeroed; `mt` is the
// valid-lag mask table of g (MaskTable<W>, usually in shared memory).  From
// two lag words up, the best pivot's step and key, written only when E
// improves, are parked in shared memory (word k at bst[k * stride]) so that
// they hold no registers during the scan (one-word walks measured faster
// keeping them in registers).  U unrolls the scan's flip loop.
template <int W, int T, int K, int PMAX, int U = 1>
__device__ __forceinline__ void run_walk(const Geometry &g, const Muls &mu, const uint32_t *mt, uint32_t *bst,
                                         int stride, uint64_t seed, uint32_t walk, uint32_t round, int walk_len,
                                         uint64_t *table, uint32_t cap, int kw64, int recheck_every, int32_t *trace,
                                         int32_t *err, WalkOut<W + 1> &out) {
  constexpr int NS = W + 1;
  WalkState<W, T> st;
  init_walk(st, g, seed, walk, round);
  {
    uint32_t slot;
    table_find(table, cap, kw64, st.key, g.D, &slot);
    table_store(table, slot, kw64, st.key, g.D);
  }
  constexpr bool kPark = W >= 2;
  int32_t bestE = st.E, moves = 0, stuck = 0, best_step = 0;
  uint32_t best_key[kPark ? 1 : NS];
  if constexpr (kPark) {
    bst[0] = 0u;
#pragma unroll
    for (int w = 0; w < NS; ++w) bst[(w + 1) * stride] = st.key[w];
  } else {
#pragma unroll
    for (int w = 0; w < NS; ++w) best_key[w] = st.key[w];
  }
  int jprev = -1;
  uint32_t plane_sum = 0;  // <= 9 * 2^26
  for (int step = 1; step <= walk_len; ++step) {
    uint32_t floor = 0;
    int chosen = -1, cdelta = 0;
    uint32_t cslot = 0;
    bool need = true;
    int tp = planes_needed(st, g);
    tp = __reduce_max_sync(__activemask(), (unsigned)tp);  // one plane count per warp (any larger count is exact)
    tp = tp < T - 3 ? T - 3 : tp;
    plane_sum += (uint32_t)tp;
    while (need) {
      uint32_t top[K];
      eval_neighbours<W, T, K, PMAX, U>(st, g, mu, mt, tp, jprev, floor, top);
#pragma unroll
      for (int r = 0; r < K; ++r) {
        if (need) {
          if (top[r] == kNone) {
            need = false;  // every neighbour not below `floor` is visited: stuck
          } else {
            const int a = key_flip(top[r]);
            uint32_t nk[NS];
#pragma unroll
            for (int w = 0; w < NS; ++w) nk[w] = st.key[w];
            xor_bit(nk, a, 1u);
            uint32_t s;
            if (!table_find(table, cap, kw64, nk, g.D, &s)) {
              need = false;
              if (s == kNone) {
                atomicOr(err, kErrOverflow);
              } else {
                chosen = a;
                cdelta = key_delta(top[r]);
                cslot = s;
              }
            }
          }
        }
      }
      if (need) floor = top[K - 1] + 1u;
    }
    if (chosen < 0) {
      stuck = 1;
      break;
    }
    apply_move(st, g, chosen, cdelta);
    table_store(table, cslot, kw64, st.key, g.D);
    jprev = chosen;
    moves = step;
    if (trace) trace[step - 1] = chosen;
    if (st.E < bestE) {
      bestE = st.E;
      if constexpr (kPark) {
        bst[0] = (uint32_t)step;
#pragma unroll
        for (int w = 0; w < NS; ++w) bst[(w + 1) * stride] = st.key[w];
      } else {
        best_step = step;
#pragma unroll
        for (int w = 0; w < NS; ++w) best_key[w] = st.key[w];
      }
    }
    if (recheck_every > 0 && (step % recheck_every) == 0 && !recheck_walk(st, g)) atomicOr(err, kErrRecheck);
  }
  out.bestE = bestE;
  out.moves = moves;
  out.stuck = stuck;
  if constexpr (kPark) {
    out.best_step = (int32_t)bst[0];
#pragma unroll
    for (int w = 0; w < NS; ++w) out.best_key[w] = bst[(w + 1) * stride];
  } else {
    out.best_step = best_step;
#pragma unroll
    for (int w = 0; w < NS; ++w) out.best_key[w] = best_key[w];
  }
  out.planes = plane_sum;
}

// One walk over the full search space (full_core.cuh): the same step loop as
// run_walk with L flips per step and the whole sequence as key; `mt` is the
// full-space mask table of L (FullMaskTable<W>).
template <int W, int T, int K>
__device__ __forceinline__ void run_walk_full(int L, const Muls &mu, const uint32_t *mt, uint64_t seed, uint32_t walk,
                                              uint32_t round, int walk_len, uint64_t *table, uint32_t cap, int kw64,
                                              int recheck_every, int32_t *trace, int32_t *err, WalkOut<W + 1> &out) {
  constexpr int NS = W + 1;
  FullState<W, T> st;
  init_full(st, L, seed, walk, round);
  {
    uint32_t slot;
    table_find(table, cap, kw64, st.bits, L, &slot);
    table_store(table, slot, kw64, st.bits, L);
  }
  int32_t bestE = st.E, best_step = 0, moves = 0, stuck = 0;
  uint32_t best_key[NS];
#pragma unroll
  for (int w = 0; w < NS; ++w) best_key[w] = st.bits[w];
  int jprev = -1;
  uint32_t plane_sum = 0;
  for (int step = 1; step <= walk_len; ++step) {
    uint32_t floor = 0;
    int chosen = -1, cdelta = 0;
    uint32_t cslot = 0;
    bool need = true;
    int tp = full_planes_needed(st, L);
    tp = __reduce_max_sync(__activemask(), (unsigned)tp);  // one plane count per warp (any larger is exact)
    tp = tp < T - 3 ? T - 3 : tp;
    plane_sum += (uint32_t)tp;
    while (need) {
      uint32_t top[K];
      full_eval<W, T, K>(st, L, mu, mt, tp, jprev, floor, top);
#pragma unroll
      for (int r = 0; r < K; ++r) {
        if (need) {
          if (top[r] == kNone) {
            need = false;  // every neighbour not below `floor` is visited: stuck
          } else {
            const int a = key_flip(top[r]);
            uint32_t nk[NS];
#pragma unroll
            for (int w = 0; w < NS; ++w) nk[w] = st.bits[w];
            xor_bit(nk, a, 1u);
            uint32_t s;
            if (!table_find(table, cap, kw64, nk, L, &s)) {
              need = false;
              if (s == kNone) {
                atomicOr(err, kErrOverflow);
              } else {
                chosen = a;
                cdelta = key_delta(top[r]);
                cslot = s;
              }
            }
          }
        }
      }
      if (need) floor = top[K - 1] + 1u;
    }
    if (chosen < 0) {
      stuck = 1;
      break;
    }
    apply_full(st, L, chosen, cdelta);
    table_store(table, cslot, kw64, st.bits, L);
    jprev = chosen;
    moves = step;
    if (trace) trace[step - 1] = chosen;
    if (st.E < bestE) {
      bestE = st.E;
      best_step = step;
#pragma unroll
      for (int w = 0; w < NS; ++w) best_key[w] = st.bits[w];
    }
    if (recheck_every > 0 && (step % recheck_every) == 0 && !recheck_full(st, L)) atomicOr(err, kErrRecheck);
  }
  out.bestE = bestE;
  out.best_step = best_step;
  out.moves = moves;
  out.stuck = stuck;
#pragma unroll
  for (int w = 0; w < NS; ++w) out.best_key[w] = best_key[w];
  out.planes = plane_sum;
}

// Storage of the incremental variant per lag-word class: C_{2i} fits int8 up
// to m = 64 (|C| <= L - 2 <= 127); Delta / 8 fits int16 while 2 m^2 + 8 m < 2^15.
template <int W>
struct IncrTypes {
  using CT = typename std::conditional<W <= 2, int8_t, int16_t>::type;
  using DT = typename std::conditional<W <= 3, int16_t, int32_t>::type;
};

template <int W>
__host__ __device__ constexpr int incr_lane_bytes() {
  return 32 * W * (int)sizeof(typename IncrTypes<W>::CT) + (32 * W + 1) * (int)sizeof(typename IncrTypes<W>::DT);
}

// One walk with the incremental neighbourhood (walk_incr.cuh): the lane's
// correlations and neighbour deltas live in shared memory `v`.
template <int W, typename CT, typename DT, int K>
__device__ __forceinline__ void run_walk_incr(const Geometry &g, const Muls &mu, const IncrView<CT, DT> &v,
                                              uint64_t seed, uint32_t walk, uint32_t round, int walk_len,
                                              uint64_t *table, uint32_t cap, int kw64, int recheck_every,
                                              int32_t *trace, int32_t *err, WalkOut<W + 1> &out) {
  constexpr int NS = W + 1;
  IncrState<W> st;
  init_incr(st, g, v, seed, walk, round);
  {
    uint32_t slot;
    table_find(table, cap, kw64, st.key, g.D, &slot);
    table_store(table, slot, kw64, st.key, g.D);
  }
  int32_t bestE = st.E, best_step = 0, moves = 0, stuck = 0;
  uint32_t best_key[NS];
#pragma unroll
  for (int w = 0; w < NS; ++w) best_key[w] = st.key[w];
  int jprev = -1;
  uint32_t top[K];
  scan_stored<W, CT, DT, K>(g, v, -1, 0u, top);
  for (int step = 1; step <= walk_len; ++step) {
    uint32_t floor = 0;
    int chosen = -1;
    uint32_t cslot = 0;
    bool need = true;
    while (need) {
#pragma unroll
      for (int r = 0; r < K; ++r) {
        if (need) {
          if (top[r] == kNone) {
            need = false;  // every neighbour not below `floor` is visited: stuck
          } else {
            const int a = key_flip(top[r]);
            uint32_t nk[NS];
#pragma unroll
            for (int w = 0; w < NS; ++w) nk[w] = st.key[w];
            xor_bit(nk, a, 1u);
            uint32_t s;
            if (!table_find(table, cap, kw64, nk, g.D, &s)) {
              need = false;
              if (s == kNone) {
                atomicOr(err, kErrOverflow);
              } else {
                chosen = a;
                cslot = s;
              }
            }
          }
        }
      }
      if (need) {
        floor = top[K - 1] + 1u;
        scan_stored<W, CT, DT, K>(g, v, jprev, floor, top);
      }
    }
    if (chosen < 0) {
      stuck = 1;
      break;
    }
    MoveData<W> md;
    apply_move_incr(st, g, v, chosen, md);
    table_store(table, cslot, kw64, st.key, g.D);
    jprev = chosen;
    moves = step;
    if (trace) trace[step - 1] = chosen;
    if (st.E < bestE) {
      bestE = st.E;
      best_step = step;
#pragma unroll
      for (int w = 0; w < NS; ++w) best_key[w] = st.key[w];
    }
    update_neighbours_fast<W, CT, DT, K>(st, g, v, md, mu, top);
    if (recheck_every > 0 && (step % recheck_every) == 0 && !recheck_incr(st, g, v)) atomicOr(err, kErrRecheck);
  }
  out.bestE = bestE;
  out.best_step = best_step;
  out.moves = moves;
  out.stuck = stuck;
#pragma unroll
  for (int w = 0; w < NS; ++w) out.best_key[w] = best_key[w];
  out.planes = 0;
}

}  // namespace psaw
