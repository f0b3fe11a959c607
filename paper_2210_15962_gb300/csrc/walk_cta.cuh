// One contiguous self-avoiding walk per CTA (Eq. 3, Algorithm 2 with the
// paper's own split: a block of threads shares one walk's neighbourhood).
// Each of the block's warps keeps what the warp-per-walk variant keeps
// (walk_warp.cuh: a register copy of the walk's state on every lane and its
// own shared mirrors of the parity classes), so moves need no exchange of
// state; the D flips of a step are split over all threads of the block
// (thread i takes flips i, i + blockDim, ...).  Each warp reduces its lanes'
// K smallest keys, the warps' lists meet in shared memory, and every thread
// takes the block's K smallest from them; warp 0 probes the visited table for
// those candidates and publishes the step's decision, which all threads read.
// Two block barriers per scan (keys published, decision published) keep the
// warps in step; every thread takes the same branches, since everything that
// decides one (the merged keys, the decision, the walk's state) is the same
// on every thread.  The trajectory is the one run_walk (one lane per walk)
// takes.
#pragma once
#include "walk_warp.cuh"

namespace psaw {

// Shared words of one CTA walk: each warp's mirrors (WarpWalkSmem, warp 0's
// parked best pivot included), the warps' K smallest keys, and the step's
// decision (outcome, flip, delta, slot or rescan floor).
template <int W>
struct CtaWalkSmem {
  static constexpr int kWarps = kWalkBlock / 32;
  static constexpr int kKeys = kWarps * WarpWalkSmem<W>::kWords;  // offset of the exchanged keys
  static constexpr int kDecision = kKeys + kWarps * kTopK;
  static constexpr int kWords = kDecision + 4;
};

// decision outcomes
constexpr uint32_t kCtaRescan = 0, kCtaStop = 1, kCtaMove = 2;

// One walk on the calling block of kWalkBlock threads (all of them call it;
// the results are the same on every thread).  `table` is the walk's visited
// table, zeroed and visible to the whole block; `mt` the mask table of g;
// `sm` the block's CtaWalkSmem<W>::kWords shared words.
template <int W, int T, int K>
__device__ void run_walk_cta(const Geometry &g, const Muls &mu, const uint32_t *mt, uint32_t *sm, uint64_t seed,
                             uint32_t walk, uint32_t round, int walk_len, uint64_t *table, uint32_t cap, int kw64,
                             int recheck_every, int32_t *trace, int32_t *err, WalkOut<W + 1> &out) {
  static_assert(K == kTopK, "the exchange buffer holds kTopK keys per warp");
  constexpr int NS = W + 1, CW = WarpWalkSmem<W>::kClsWords, P = CtaWalkSmem<W>::kWarps;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t *wsm = sm + warp * WarpWalkSmem<W>::kWords;  // this warp's mirrors
  uint32_t *keys = sm + CtaWalkSmem<W>::kKeys;          // [warp][K]
  uint32_t *dec = sm + CtaWalkSmem<W>::kDecision;
  uint32_t *park = sm + 4 * CW;  // warp 0's: best step, then the best key
  WalkState<W, T> st;
  init_walk(st, g, seed, walk, round);
  for (int k = lane; k < 4 * CW; k += 32) wsm[k] = 0u;  // the zero pads
  __syncwarp();
  warp_publish_classes(st, wsm, lane);
  if (tid == 0) {
    uint32_t slot;
    table_find(table, cap, kw64, st.key, g.D, &slot);
    table_store(table, slot, kw64, st.key, g.D);
    park[0] = 0u;
#pragma unroll
    for (int w = 0; w < NS; ++w) park[1 + w] = st.key[w];
  }
  __syncthreads();
  int32_t bestE = st.E, moves = 0, stuck = 0;
  int jprev = -1;
  uint32_t plane_sum = 0;
  for (int step = 1; step <= walk_len; ++step) {
    const int tp0 = planes_needed(st, g);  // the same on every thread
    const int tp = tp0 < T - 3 ? T - 3 : tp0;
    plane_sum += (uint32_t)tp;
    uint32_t floor = 0;
    int chosen = -1, cdelta = 0;
    uint32_t cslot = 0;
    bool decided = false;
    while (!decided) {
      uint32_t wtop[K];
      warp_scan<W, T, K>(st, g, mu, mt, wsm, tid, kWalkBlock, tp, jprev, floor, wtop);
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < K; ++r) keys[warp * K + r] = wtop[r];
      }
      __syncthreads();  // every warp's keys are published
      uint32_t ctop[K];
#pragma unroll
      for (int r = 0; r < K; ++r) ctop[r] = kNone;
#pragma unroll
      for (int i = 0; i < P * K; ++i) top_insert(ctop, keys[i]);
      if (warp == 0) {
        // lane r < K probes candidate r; the first candidate in key order that
        // is absent (no more neighbours: stuck) or unvisited decides the step
        uint32_t cand = kNone;
#pragma unroll
        for (int r = 0; r < K; ++r) cand = lane == r ? ctop[r] : cand;
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
        uint32_t c = kNone, sl = kNone;
        if (hits) {
          const int r = __ffs(hits) - 1;
          c = __shfl_sync(0xFFFFFFFFu, cand, r);
          sl = __shfl_sync(0xFFFFFFFFu, s, r);
        }
        if (lane == 0) {
          if (!hits) {
            dec[0] = kCtaRescan;
            dec[3] = ctop[K - 1] + 1u;  // every candidate visited: rescan above them
          } else if (c == kNone || sl == kNone) {
            if (c != kNone) atomicOr(err, kErrOverflow);
            dec[0] = kCtaStop;
          } else {
            dec[0] = kCtaMove;
            dec[1] = (uint32_t)key_flip(c);
            dec[2] = (uint32_t)key_delta(c);
            dec[3] = sl;
          }
        }
      }
      __syncthreads();  // the decision is published; the keys may be overwritten
      const uint32_t kind = dec[0];
      if (kind == kCtaRescan) {
        floor = dec[3];
      } else {
        decided = true;
        if (kind == kCtaMove) {
          chosen = (int)dec[1];
          cdelta = (int)dec[2];
          cslot = dec[3];
        }
      }
    }
    if (chosen < 0) {
      stuck = 1;
      break;
    }
    warp_apply_move(st, g, wsm, lane, chosen, cdelta);
    if (tid == 0) {
      table_store(table, cslot, kw64, st.key, g.D);
      if (trace) trace[step - 1] = chosen;
    }
    jprev = chosen;
    moves = step;
    if (st.E < bestE) {
      bestE = st.E;
      if (tid == 0) {
        park[0] = (uint32_t)step;
#pragma unroll
        for (int w = 0; w < NS; ++w) park[1 + w] = st.key[w];
      }
    }
    if (recheck_every > 0 && (step % recheck_every) == 0 && tid == 0 && !recheck_walk(st, g))
      atomicOr(err, kErrRecheck);
  }
  __syncthreads();  // thread 0's last parked pivot is visible
  out.bestE = bestE;
  out.moves = moves;
  out.stuck = stuck;
  out.best_step = (int32_t)park[0];
#pragma unroll
  for (int w = 0; w < NS; ++w) out.best_key[w] = park[1 + w];
  out.planes = plane_sum;
}

}  // namespace psaw
