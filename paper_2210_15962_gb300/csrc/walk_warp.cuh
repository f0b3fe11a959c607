// One contiguous self-avoiding walk per warp (Eq. 3, Algorithm 2): the 32
// lanes split the D flips of every step, as the paper's block of threads
// splits them, instead of one lane owning a whole walk.  Every lane keeps a
// copy of the walk's state (walk_core.cuh: the parity classes, the digit
// planes of the even correlations, the key and E) and applies every move to
// it, so the state never has to be exchanged; the class bit arrays and their
// bit reversals are mirrored in shared memory so that each lane can cut the
// lag windows of its own flips at any position.  Each lane keeps the K
// smallest keys of its flips; the warp merges them by K minimum reductions
// (ties go to the lowest flip: the flip index is the key's low byte), lanes
// 0..K-1 probe the visited table for the K candidates at once, and the first
// unvisited candidate in key order is the move.  The trajectory is the one
// run_walk (one lane per walk) takes.
#pragma once
#include "walk_device.cuh"

namespace psaw {

// Shared words of one warp: the two parity classes and their bit reversals,
// each padded with zero words so that a window cut at any flip reads zeros
// past the ends, then the parked best pivot (step, key words).
template <int W>
struct WarpWalkSmem {
  static constexpr int kClsWords = 2 * W + 2;     // >= (W + 1) + ceil(W / 2) + 1
  static constexpr int kWords = 4 * kClsWords + W + 2;
};

// Copy the classes and their reversals (as 32 (W+1)-bit numbers) to shared memory.
template <int W, int T>
__device__ __forceinline__ void warp_publish_classes(const WalkState<W, T> &st, uint32_t *sm, int lane) {
  constexpr int NS = W + 1, CW = WarpWalkSmem<W>::kClsWords;
  if (lane < NS) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      uint32_t c = 0, r = 0;
#pragma unroll
      for (int w = 0; w < NS; ++w) {
        c |= st.cls[q][w] & sel_mask(w == lane);
        r |= st.cls[q][w] & sel_mask(NS - 1 - w == lane);
      }
      sm[q * CW + lane] = c;
      sm[(2 + q) * CW + lane] = brev32(r);
    }
  }
  __syncwarp();
}

// The move of flip a on every lane's copy of the walk: its windows cut from
// the shared mirrors (as the scan cuts them), the planes' update and the bit
// flips in registers; then lane 0 flips the same bits in the mirrors (the
// position, its Eq. 2 mirror, and their places in the reversal).
template <int W, int T>
__device__ __forceinline__ void warp_apply_move(WalkState<W, T> &st, const Geometry &g, uint32_t *sm, int lane,
                                                int a, int delta) {
  constexpr int NS = W + 1, CW = WarpWalkSmem<W>::kClsWords;
  const int q = a & 1, t = a >> 1;
  const uint32_t *C = sm + q * CW;
  const uint32_t *R = sm + (2 + q) * CW;
  uint32_t F[W], X[W];
  const int of = (t + 1) >> 5, sf = (t + 1) & 31;
#pragma unroll
  for (int w = 0; w < W; ++w) F[w] = fshr(C[of + w], C[of + w + 1], (uint32_t)sf);
  const int u = 32 * NS - t, ob = u >> 5, sb = u & 31;
#pragma unroll
  for (int w = 0; w < W; ++w) X[w] = w < x_words<W>() ? fshr(R[ob + w], R[ob + w + 1], (uint32_t)sb) : 0u;
  const uint32_t ba = (C[t >> 5] >> (t & 31)) & 1u;
  move_planes(st, g, a, delta, ba, F, X);
  move_bits(st, g, a);
  __syncwarp();  // every lane has read the mirrors before lane 0 changes them
  if (lane == 0) {
    uint32_t *Cw = sm + q * CW;
    uint32_t *Rw = sm + (2 + q) * CW;
    const int r = 32 * NS - 1 - t;
    Cw[t >> 5] ^= 1u << (t & 31);
    Rw[r >> 5] ^= 1u << (r & 31);
    if (a != g.c) {
      const int k = (g.L - 1 - a - q) >> 1, rk = 32 * NS - 1 - k;
      Cw[k >> 5] ^= 1u << (k & 31);
      Rw[rk >> 5] ^= 1u << (rk & 31);
    }
  }
  __syncwarp();
}

// The K smallest keys of the flips this thread owns in class q (t = first,
// first + stride, ...: a lane of a warp that owns the walk takes every 32nd
// flip, a thread of a CTA that owns it every blockDim-th), as
// eval_neighbours_tp computes them for one flip each.
template <int W, int T, int TP, int K, bool RESCAN>
__device__ __forceinline__ void warp_scan_class(const WalkState<W, T> &st, const Geometry &g, const Muls &mu,
                                                const uint32_t *mt, const uint32_t *sm, int q, int first,
                                                int stride, int jprev, uint32_t floor, uint32_t (&top)[K]) {
  using MT = MaskTable<W>;
  constexpr int NS = W + 1, CW = WarpWalkSmem<W>::kClsWords;
  const int Nq = g.D - q;
  const int n = Nq - 2;
  const bool has_centre = (g.c & 1) == q;
  const int nloop = (q ? g.D / 2 : (g.D + 1) / 2) - (has_centre ? 1 : 0);
  const int tprev = (jprev >= 0 && (jprev & 1) == q) ? (jprev >> 1) : -1;
  const int tpair = (g.c - q + 2) / 3;
  const uint32_t *C = sm + q * CW;
  const uint32_t *R = sm + (2 + q) * CW;
  const uint32_t *rows = mt + (size_t)q * MT::kRows * MT::kRowWords;
  const int tend = nloop + (has_centre ? 1 : 0);
  for (int t = first; t < tend; t += stride) {
    // y window: class bits t+1, t+2, ...; x window: bits t-1, t-2, ...
    // (the reversal R holds class bit 32 NS - 1 - k at bit k)
    uint32_t F[W], B[W];
    const int of = (t + 1) >> 5, sf = (t + 1) & 31;
#pragma unroll
    for (int w = 0; w < W; ++w) F[w] = fshr(C[of + w], C[of + w + 1], (uint32_t)sf);
    const int u = 32 * NS - t, ob = u >> 5, sb = u & 31;
#pragma unroll
    for (int w = 0; w < W; ++w) B[w] = w < x_words<W>() ? fshr(R[ob + w], R[ob + w + 1], (uint32_t)sb) : 0u;
    const uint32_t ba = (C[t >> 5] >> (t & 31)) & 1u;
    uint32_t Vx[W], Vye[W];
    load_mask_row<W>(rows + (size_t)t * MT::kRowWords, Vx, Vye);
    const int a = 2 * t + q;
    uint32_t x;
    if (t < nloop) {
      const int nxy = t - (t >= tpair ? 1 : 0);
      x = flip_key<W, T, TP, false, -1, -1, true>(st, mu, B, F, Vx, Vye, ba, key_base<TP>(a, n, nxy),
                                                  key_diff<TP>(n, nxy), t, Nq);
      x = (t == tprev || (RESCAN && x < floor)) ? kNone : x;
    } else {  // the centre: n = |Vx| = t, no y side
      x = flip_key<W, T, TP, true, -1, -1, true>(st, mu, B, F, Vx, Vye, ba, key_base<TP>(a, t, 0),
                                                 key_diff<TP>(t, 0), t, Nq);
      x = (a == jprev || (RESCAN && x < floor)) ? kNone : x;
    }
    top_insert(top, x);
  }
}

template <int W, int T, int TP, int K, bool RESCAN>
__device__ __forceinline__ void warp_scan_tp(const WalkState<W, T> &st, const Geometry &g, const Muls &mu,
                                             const uint32_t *mt, const uint32_t *sm, int first, int stride,
                                             int jprev, uint32_t floor, uint32_t (&top)[K]) {
#pragma unroll
  for (int r = 0; r < K; ++r) top[r] = kNone;
  warp_scan_class<W, T, TP, K, RESCAN>(st, g, mu, mt, sm, 0, first, stride, jprev, floor, top);
  warp_scan_class<W, T, TP, K, RESCAN>(st, g, mu, mt, sm, 1, first, stride, jprev, floor, top);
}

// The warp's K smallest keys in order (warp-uniform), from each lane's K smallest.
template <int K>
__device__ __forceinline__ void warp_merge_top(uint32_t (&top)[K], uint32_t (&wtop)[K]) {
#pragma unroll
  for (int r = 0; r < K; ++r) {
    const uint32_t m = __reduce_min_sync(0xFFFFFFFFu, top[0]);
    wtop[r] = m;
    if (top[0] == m && m != kNone) {  // keys are distinct: exactly one lane owns m
#pragma unroll
      for (int i = 0; i + 1 < K; ++i) top[i] = top[i + 1];
      top[K - 1] = kNone;
    }
  }
}

// The warp's K smallest keys of the flips its threads own (first, stride as
// in warp_scan_class), in order and warp-uniform.
template <int W, int T, int K>
__device__ __forceinline__ void warp_scan(const WalkState<W, T> &st, const Geometry &g, const Muls &mu,
                                          const uint32_t *mt, const uint32_t *sm, int first, int stride, int tp,
                                          int jprev, uint32_t floor, uint32_t (&wtop)[K]) {
  constexpr int T3 = T - 3 >= 2 ? T - 3 : 2;
  uint32_t top[K];
  if (floor == 0) {
    if (tp >= T) warp_scan_tp<W, T, T, K, false>(st, g, mu, mt, sm, first, stride, jprev, 0u, top);
    else if (tp == T - 1) warp_scan_tp<W, T, T - 1, K, false>(st, g, mu, mt, sm, first, stride, jprev, 0u, top);
    else if (tp == T - 2) warp_scan_tp<W, T, T - 2, K, false>(st, g, mu, mt, sm, first, stride, jprev, 0u, top);
    else warp_scan_tp<W, T, T3, K, false>(st, g, mu, mt, sm, first, stride, jprev, 0u, top);
  } else {
    if (tp >= T) warp_scan_tp<W, T, T, K, true>(st, g, mu, mt, sm, first, stride, jprev, floor, top);
    else if (tp == T - 1) warp_scan_tp<W, T, T - 1, K, true>(st, g, mu, mt, sm, first, stride, jprev, floor, top);
    else if (tp == T - 2) warp_scan_tp<W, T, T - 2, K, true>(st, g, mu, mt, sm, first, stride, jprev, floor, top);
    else warp_scan_tp<W, T, T3, K, true>(st, g, mu, mt, sm, first, stride, jprev, floor, top);
  }
  warp_merge_top<K>(top, wtop);
}

// One walk on one warp (all 32 lanes call it; the results are the same on
// every lane).  `table` is the walk's visited table, zeroed; `mt` the mask
// table of g; `sm` the warp's WarpWalkSmem<W>::kWords shared words.
template <int W, int T, int K>
__device__ void run_walk_warp(const Geometry &g, const Muls &mu, const uint32_t *mt, uint32_t *sm, uint64_t seed,
                              uint32_t walk, uint32_t round, int walk_len, uint64_t *table, uint32_t cap, int kw64,
                              int recheck_every, int32_t *trace, int32_t *err, WalkOut<W + 1> &out) {
  constexpr int NS = W + 1, CW = WarpWalkSmem<W>::kClsWords;
  const int lane = threadIdx.x & 31;
  WalkState<W, T> st;
  init_walk(st, g, seed, walk, round);
  for (int k = lane; k < 4 * CW; k += 32) sm[k] = 0u;  // the zero pads
  __syncwarp();
  warp_publish_classes(st, sm, lane);
  uint32_t *park = sm + 4 * CW;  // best step, then the best key
  if (lane == 0) {
    uint32_t slot;
    table_find(table, cap, kw64, st.key, g.D, &slot);
    table_store(table, slot, kw64, st.key, g.D);
    park[0] = 0u;
#pragma unroll
    for (int w = 0; w < NS; ++w) park[1 + w] = st.key[w];
  }
  __syncwarp();
  int32_t bestE = st.E, moves = 0, stuck = 0;
  int jprev = -1;
  uint32_t plane_sum = 0;
  for (int step = 1; step <= walk_len; ++step) {
    const int tp0 = planes_needed(st, g);  // the same on every lane
    const int tp = tp0 < T - 3 ? T - 3 : tp0;
    plane_sum += (uint32_t)tp;
    uint32_t floor = 0;
    int chosen = -1, cdelta = 0;
    uint32_t cslot = 0;
    bool decided = false;
    while (!decided) {
      uint32_t wtop[K];
      warp_scan<W, T, K>(st, g, mu, mt, sm, lane, 32, tp, jprev, floor, wtop);
      // lane r < K probes candidate r; the first candidate in key order that is
      // absent (no more neighbours: stuck) or unvisited decides the step
      uint32_t cand = kNone;
#pragma unroll
      for (int r = 0; r < K; ++r) cand = lane == r ? wtop[r] : cand;
      bool stop_here = false;
      uint32_t s = kNone;
      if (lane < K) {
        if (cand == kNone) {
          stop_here = true;
        } else {
          uint32_t nk[NS];
#pragma unroll
          for (int w = 0; w < NS; ++w) nk[w] = st.key[w];
          xor_bit(nk, key_flip(cand), 1u);
          stop_here = !table_find(table, cap, kw64, nk, g.D, &s);
        }
      }
      const uint32_t hits = __ballot_sync(0xFFFFFFFFu, stop_here);
      if (hits) {
        const int r = __ffs(hits) - 1;
        const uint32_t c = __shfl_sync(0xFFFFFFFFu, cand, r);
        const uint32_t sl = __shfl_sync(0xFFFFFFFFu, s, r);
        decided = true;
        if (c != kNone) {
          if (sl == kNone) {
            if (lane == 0) atomicOr(err, kErrOverflow);
          } else {
            chosen = key_flip(c);
            cdelta = key_delta(c);
            cslot = sl;
          }
        }
      } else {
        floor = wtop[K - 1] + 1u;  // every candidate visited: rescan above them
      }
    }
    if (chosen < 0) {
      stuck = 1;
      break;
    }
    warp_apply_move(st, g, sm, lane, chosen, cdelta);
    if (lane == 0) {
      table_store(table, cslot, kw64, st.key, g.D);
      if (trace) trace[step - 1] = chosen;
    }
    __syncwarp();
    jprev = chosen;
    moves = step;
    if (st.E < bestE) {
      bestE = st.E;
      if (lane == 0) {
        park[0] = (uint32_t)step;
#pragma unroll
        for (int w = 0; w < NS; ++w) park[1 + w] = st.key[w];
      }
    }
    if (recheck_every > 0 && (step % recheck_every) == 0 && lane == 0 && !recheck_walk(st, g))
      atomicOr(err, kErrRecheck);
  }
  __syncwarp();
  out.bestE = bestE;
  out.moves = moves;
  out.stuck = stuck;
  out.best_step = (int32_t)park[0];
#pragma unroll
  for (int w = 0; w < NS; ++w) out.best_key[w] = park[1 + w];
  out.planes = plane_sum;
}

}  // namespace psaw
