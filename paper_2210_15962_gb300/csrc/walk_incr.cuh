// Incremental neighbourhood evaluation of one contiguous self-avoiding walk
// (Eq. 1-3, Algorithm 2): instead of recomputing every neighbour's energy
// change from the correlations at every step, each lane keeps the D values
// Delta_j and the m correlations C_{2i} of its walk in shared memory and
// updates them after each move.
//
// With u_i(j) = s_a (s_{a-2i} [x-side] + s_{a+2i} [y-side]) the per-lag factor
// of flip j (position a; see walk_core.cuh), Delta_j = -8 u(j).C + 16 |u(j)|^2.
// A move j* (position a*) changes C by -4 d, d = u(j*), negates Delta_{j*},
// and changes u(j) of every other flip by eps(j) = u'(j) - u(j), which is
// nonzero at no more than two lags (the lags at which a* or its mirror sit in
// j's windows, same parity class only).  Expanding the squares gives, exactly,
//   Delta'_j = Delta_j + 32 u'(j).d + 8 sum_i eps_i (-C'_i - 4 d_i + 4 u'_i - 2 eps_i)
// with C' = C - 4d the new correlations.  The dense term u'(j).d is a dot
// product of two lag vectors with entries in {-2..2}: four masked XOR
// popcounts per 32 lags (x/y side of j against x/y side of j*), against
// 4 TP masked XORs + TP popcounts of a full evaluation.
#pragma once
#include "walk_core.cuh"

namespace psaw {

// Bits of a walk (the correlations and neighbour deltas live in shared memory).
template <int W>
struct IncrState {
  static constexpr int NS = W + 1;
  uint32_t cls[2][NS];  // cls[q] bit t = b(2t + q)
  uint32_t key[NS];     // key bit j = b(j), j < D
  int32_t E;
};

// One lane's shared-memory arrays: C_{2i} at C[(i-1) * stride] (i = 1..m) and
// Delta_j at Dl[j * stride] (j = 0..D-1).  With 16-bit delta storage the
// value stored is Delta / 8 (Delta is always a multiple of 8).
template <typename CT, typename DT>
struct IncrView {
  CT *C;
  DT *Dl;
  int stride;
  LABS_HD int getC(int i) const { return (int)C[(size_t)(i - 1) * stride]; }
  LABS_HD void setC(int i, int v) { C[(size_t)(i - 1) * stride] = (CT)v; }
  LABS_HD int getD(int j) const {
    return sizeof(DT) == 2 ? 8 * (int)Dl[(size_t)j * stride] : (int)Dl[(size_t)j * stride];
  }
  LABS_HD void setD(int j, int v) { Dl[(size_t)j * stride] = (DT)(sizeof(DT) == 2 ? v / 8 : v); }
};

// P_1 of Eq. 3 (same stream layout as init_walk) and its bits.
template <int W>
LABS_HD void init_bits(IncrState<W> &st, const Geometry &g, uint64_t seed, uint32_t walk, uint32_t round) {
  constexpr int NS = W + 1;
  uint32_t blk[4] = {0, 0, 0, 0};
#pragma unroll
  for (int w = 0; w < NS; ++w) {
    if ((w & 3) == 0) {
      blk[0] = walk;
      blk[1] = round;
      blk[2] = (uint32_t)(w >> 2);
      blk[3] = 0;
      philox4x32_10(blk, (uint32_t)seed, (uint32_t)(seed >> 32));
    }
    st.key[w] = blk[w & 3] & low_mask_word(g.D, w);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int w = 0; w < NS; ++w) st.cls[q][w] = 0;
  for (int a = 0; a < g.L; ++a) {
    uint32_t b;
    if (a < g.D) {
      b = get_bit(st.key, a);
    } else {
      const int i = a - g.c;  // s_{c+i} = (-1)^i s_{c-i}
      b = get_bit(st.key, g.c - i) ^ (uint32_t)(i & 1);
    }
    if (a & 1) xor_bit(st.cls[1], a >> 1, b);
    else xor_bit(st.cls[0], a >> 1, b);
  }
}

// C_{2i}, i = 1..m, by XOR + popc over the class arrays (as next_even_correlation).
template <int W, typename F>
LABS_HD void for_each_correlation(const IncrState<W> &st, const Geometry &g, F f) {
  constexpr int NS = W + 1;
  uint32_t sh[2][NS];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int w = 0; w < NS; ++w) sh[q][w] = st.cls[q][w];
  for (int i = 1; i <= g.m; ++i) {
    int C = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
      for (int w = 0; w < NS; ++w) sh[q][w] = fshr(sh[q][w], (w + 1 < NS) ? sh[q][w + 1] : 0u, 1u);
      const int pairs = g.N[q] - i;
      if (pairs > 0) {
        int dis = 0;
#pragma unroll
        for (int w = 0; w < NS; ++w) dis += (int)popc32((st.cls[q][w] ^ sh[q][w]) & low_mask_word(pairs, w));
        C += pairs - 2 * dis;
      }
    }
    f(i, C);
  }
}

// Lag windows of the flip at class index t of class q (bit i-1 = lag i):
// X bits b(a-2i), Y bits b(a+2i), Vx valid x lags, Vy valid y lags without the
// flip's own mirror pair (empty for the centre); sa = b(a).
template <int W>
struct FlipWindows {
  uint32_t X[W], Y[W], Vx[W], Vy[W];
  uint32_t ba;
};

template <int W>
LABS_HD void flip_windows(const IncrState<W> &st, const Geometry &g, int a, FlipWindows<W> &fw) {
  constexpr int NS = W + 1;
  const int q = a & 1, t = a >> 1;
  const int Nq = g.D - q;
  const bool centre = (a == g.c);
  uint32_t cq[NS];
  const uint32_t mq = sel_mask(q != 0);
#pragma unroll
  for (int w = 0; w < NS; ++w) cq[w] = (st.cls[1][w] & mq) | (st.cls[0][w] & ~mq);
  fw.ba = get_bit(cq, t);
  uint32_t R[NS];
  shr_dyn(fw.Y, cq, t + 1);
#pragma unroll
  for (int w = 0; w < NS; ++w) R[w] = brev32(cq[NS - 1 - w]);
  shr_dyn(fw.X, R, 32 * NS - t);
  const int i0 = g.c - a;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    fw.Vx[w] = low_mask_word(t, w);
    uint32_t vy = centre ? 0u : low_mask_word(Nq - 1 - t, w);
    if (!centre && ((i0 - 1) >> 5) == w) vy &= ~(1u << ((i0 - 1) & 31));
    fw.Vy[w] = vy;
  }
}

// u_i of a flip from its windows, at lag i (1 <= i <= m)
template <int W>
LABS_HD int u_at(const FlipWindows<W> &fw, int i) {
  const int p = i - 1;
  const uint32_t xv = get_bit(fw.Vx, p), yv = get_bit(fw.Vy, p);
  const int x = xv ? (get_bit(fw.X, p) ? -1 : 1) : 0;
  const int y = yv ? (get_bit(fw.Y, p) ? -1 : 1) : 0;
  return (fw.ba ? -1 : 1) * (x + y);
}

// Delta_j from scratch from the stored correlations (first step of a walk,
// and the recheck): Delta = sum_i (-8 u_i C_i + 16 u_i^2).
template <int W, typename CT, typename DT>
LABS_HD int full_delta(const IncrState<W> &st, const Geometry &g, const IncrView<CT, DT> &v, int a) {
  FlipWindows<W> fw;
  flip_windows(st, g, a, fw);
  int d = 0;
  for (int i = 1; i <= g.m; ++i) {
    const int u = u_at(fw, i);
    d += -8 * u * v.getC(i) + 16 * u * u;
  }
  return d;
}

// Start a walk: bits, C, E, and every Delta_j; the K smallest keys go to top.
template <int W, typename CT, typename DT>
LABS_HD void init_incr(IncrState<W> &st, const Geometry &g, const IncrView<CT, DT> &v, uint64_t seed, uint32_t walk,
                       uint32_t round) {
  init_bits(st, g, seed, walk, round);
  int32_t E = 0;
  for_each_correlation(st, g, [&](int i, int C) {
    E += C * C;
    v.C[(size_t)(i - 1) * v.stride] = (CT)C;
  });
  st.E = E;
  for (int a = 0; a < g.D; ++a) {
    IncrView<CT, DT> vv = v;
    vv.setD(a, full_delta(st, g, v, a));
  }
}

// The move data of j*: its windows in the old sequence and its position.
template <int W>
struct MoveData {
  FlipWindows<W> fw;  // of j* before the move
  int a, q, t, Nq;
  uint32_t sa_old;     // b(a*) before the move
  uint32_t smir_new;   // b(mirror(a*)) after the move
};

// Apply move a*: flip the bits, E += Delta_{a*}, C_i -= 4 d_i, Delta_{a*} := -Delta_{a*}.
template <int W, typename CT, typename DT>
LABS_HD void apply_move_incr(IncrState<W> &st, const Geometry &g, const IncrView<CT, DT> &v, int a, MoveData<W> &md) {
  constexpr int NS = W + 1;
  flip_windows(st, g, a, md.fw);
  md.a = a;
  md.q = a & 1;
  md.t = a >> 1;
  md.Nq = g.D - md.q;
  md.sa_old = md.fw.ba;
  const int dA = v.getD(a);
  st.E += dA;
  IncrView<CT, DT> vv = v;
  vv.setD(a, -dA);
  // C_i -= 4 u_i(j*): walk the lags with shifting copies of the windows
  uint32_t X[W], Y[W], Vx[W], Vy[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    X[w] = md.fw.X[w];
    Y[w] = md.fw.Y[w];
    Vx[w] = md.fw.Vx[w];
    Vy[w] = md.fw.Vy[w];
  }
  const int sgn = md.fw.ba ? -1 : 1;
  for (int i = 1; i <= g.m; ++i) {
    const int x = (Vx[0] & 1u) ? ((X[0] & 1u) ? -1 : 1) : 0;
    const int y = (Vy[0] & 1u) ? ((Y[0] & 1u) ? -1 : 1) : 0;
    const int u = sgn * (x + y);
    if (u) vv.setC(i, v.getC(i) - 4 * u);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t nx = (w + 1 < W) ? X[w + 1] : 0u, ny = (w + 1 < W) ? Y[w + 1] : 0u;
      const uint32_t nvx = (w + 1 < W) ? Vx[w + 1] : 0u, nvy = (w + 1 < W) ? Vy[w + 1] : 0u;
      X[w] = fshr(X[w], nx, 1u);
      Y[w] = fshr(Y[w], ny, 1u);
      Vx[w] = fshr(Vx[w], nvx, 1u);
      Vy[w] = fshr(Vy[w], nvy, 1u);
    }
  }
  // flip the bits (a* and its mirror)
  uint32_t cq[NS];
  const uint32_t mq = sel_mask(md.q != 0);
#pragma unroll
  for (int w = 0; w < NS; ++w) cq[w] = (st.cls[1][w] & mq) | (st.cls[0][w] & ~mq);
  const bool centre = (a == g.c);
  xor_bit(cq, md.t, 1u);
  const int tm = (g.L - 1 - a - md.q) >> 1;
  if (!centre) xor_bit(cq, tm, 1u);
#pragma unroll
  for (int w = 0; w < NS; ++w) {
    st.cls[0][w] = (st.cls[0][w] & mq) | (cq[w] & ~mq);
    st.cls[1][w] = (cq[w] & mq) | (st.cls[1][w] & ~mq);
  }
  xor_bit(st.key, a, 1u);
  md.smir_new = get_bit(cq, tm);
}

// u_i of a flip at lag i from scan-time windows (B: x bits, F: y bits, masks
// Vx and Vy minus the pair hole Pm; y side empty for the centre).
template <int W>
LABS_HD int u_scan(const uint32_t (&B)[W], const uint32_t (&F)[W], const uint32_t (&Vx)[W], const uint32_t (&Vy)[W],
                   const uint32_t (&Pm)[W], bool centre, uint32_t ba, int i) {
  const int p = i - 1;
  const int x = get_bit(Vx, p) ? (get_bit(B, p) ? -1 : 1) : 0;
  const int y = (!centre && get_bit(Vy, p) && !get_bit(Pm, p)) ? (get_bit(F, p) ? -1 : 1) : 0;
  return (ba ? -1 : 1) * (x + y);
}

// The update pass after a move: Delta'_j for every flip j != a*, stored back,
// and the K smallest packed keys excluding a* (the new previous pivot).  Flips
// are scanned class by class with windows that advance one lag per flip.  Per
// 32 lags the flip's x/y sides are dotted with j*'s
// x/y sides by four masked XOR popcounts (sides of the flip with no valid lag
// in a word are skipped: the same for every lane); the mask sizes come from
// their prefix structure; flips of j*'s parity class add the sparse terms.
template <int W, typename CT, typename DT, int K>
LABS_HD void update_neighbours_fast(const IncrState<W> &st, const Geometry &g, const IncrView<CT, DT> &v,
                                    const MoveData<W> &md, const Muls &mu, uint32_t (&top)[K]) {
#pragma unroll
  for (int r = 0; r < K; ++r) top[r] = kNone;
  const int sstar = md.sa_old ? -1 : 1;
  IncrView<CT, DT> vv = v;
  const int lx_s = md.t;
  const int ly_s = (md.a == g.c) ? 0 : md.Nq - 1 - md.t;
  const int pair_s = (md.a == g.c) ? -1 : g.c - md.a;
  const int s_astar_new = md.sa_old ? 1 : -1;
  const int s_mir_new = md.smir_new ? -1 : 1;
  const int amir = g.L - 1 - md.a;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int Nq = g.N[q];
    uint32_t F[W], B[W], Vx[W], Vy[W], Pm[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      F[w] = fshr(st.cls[q][w], st.cls[q][w + 1], 1u);
      B[w] = 0;
      Vx[w] = 0;
      Vy[w] = low_mask_word(Nq - 1, w);
      Pm[w] = ((g.c - q - 1) >> 5) == w ? (1u << ((g.c - q - 1) & 31)) : 0u;
    }
    uint32_t ba = st.cls[q][0] & 1u;
    for (int t = 0; t < g.nfree[q]; ++t) {
      const int a = 2 * t + q;
      const bool centre = (a == g.c);
      if (a != md.a) {
        const int lx = t, ly = centre ? 0 : Nq - 1 - t, pr = centre ? -1 : g.c - a;
        // sizes of the four mask intersections (prefixes minus the pair holes)
        int ncnt = 0;
        {
          const int la[2] = {lx, ly}, pa[2] = {-1, pr}, lb[2] = {lx_s, ly_s}, pb[2] = {-1, pair_s};
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int z = 0; z < 2; ++z) {
              const int mm = la[u] < lb[z] ? la[u] : lb[z];
              int n = mm;
              if (pa[u] >= 1 && pa[u] <= mm) --n;
              if (pb[z] >= 1 && pb[z] <= mm && pb[z] != pa[u]) --n;
              ncnt += n;
            }
        }
        uint32_t xcnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          constexpr bool kSkip = W <= kSkipMaxWords;
          const bool xa = kSkip ? (t > 32 * w) : true;
          const bool ya = kSkip ? (!centre && (Nq - 1 - t > 32 * w)) : !centre;
          if (xa) {
            xcnt += popc32(Vx[w] & md.fw.Vx[w] & (B[w] ^ md.fw.X[w]));
            xcnt += popc32(Vx[w] & md.fw.Vy[w] & (B[w] ^ md.fw.Y[w]));
          }
          if (ya) {
            const uint32_t vy = Vy[w] & ~Pm[w];
            xcnt += popc32(vy & md.fw.Vx[w] & (F[w] ^ md.fw.X[w]));
            xcnt += popc32(vy & md.fw.Vy[w] & (F[w] ^ md.fw.Y[w]));
          }
        }
        const int sa = ba ? -1 : 1;
        int dnew = v.getD(a) + 32 * sa * sstar * (ncnt - 2 * (int)xcnt);
        if (q == md.q) {
          // lag of a*: y side of a (a < a*) or x side (a > a*)
          {
            const int i = (a < md.a) ? (md.a - a) >> 1 : (a - md.a) >> 1;
            const int eps = 2 * sa * s_astar_new;
            const int up = u_scan(B, F, Vx, Vy, Pm, centre, ba, i);
            const int d = u_at(md.fw, i);
            dnew += 8 * eps * (-v.getC(i) - 4 * d + 4 * up - 2 * eps);
          }
          // lag of a*'s mirror (y side), unless a* or a is the centre
          if (md.a != g.c && !centre) {
            const int i = (amir - a) >> 1;
            const int eps = 2 * sa * s_mir_new;
            const int up = u_scan(B, F, Vx, Vy, Pm, centre, ba, i);
            const int d = u_at(md.fw, i);
            dnew += 8 * eps * (-v.getC(i) - 4 * d + 4 * up - 2 * eps);
          }
        }
        vv.setD(a, dnew);
        top_insert(top, imad((uint32_t)(dnew + kDeltaBias), 256u, (uint32_t)a));
      }
      // advance the windows and masks by one lag
      const uint32_t ba_next = F[0] & 1u;
#pragma unroll
      for (int w = W - 1; w >= 1; --w) {
        B[w] = imadhi(B[w - 1], mu.two, imad(B[w], mu.two, 0u));
        Vx[w] = imadhi(Vx[w - 1], mu.two, imad(Vx[w], mu.two, 0u));
      }
      B[0] = imad(B[0], mu.two, ba);
      Vx[0] = imad(Vx[0], mu.two, 1u);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        F[w] = imadhi(F[w], mu.h31, (w + 1 < W) ? imad(F[w + 1], mu.h31, 0u) : 0u);
        Vy[w] = imadhi(Vy[w], mu.h31, (w + 1 < W) ? imad(Vy[w + 1], mu.h31, 0u) : 0u);
        Pm[w] = imadhi(Pm[w], mu.h30, (w + 1 < W) ? imad(Pm[w + 1], mu.h30, 0u) : 0u);
      }
      ba = ba_next;
    }
  }
}

// Candidates from the stored deltas (a rescan above `floor`, or after init).
template <int W, typename CT, typename DT, int K>
LABS_HD void scan_stored(const Geometry &g, const IncrView<CT, DT> &v, int jprev, uint32_t floor, uint32_t (&top)[K]) {
#pragma unroll
  for (int r = 0; r < K; ++r) top[r] = kNone;
  for (int a = 0; a < g.D; ++a) {
    uint32_t x = ((uint32_t)(v.getD(a) + kDeltaBias) << 8) | (uint32_t)a;
    x = (a == jprev || x < floor) ? kNone : x;
    top_insert(top, x);
  }
}

// Debug recheck: C from XOR + popc, E from Eq. 1, every stored Delta from scratch.
template <int W, typename CT, typename DT>
LABS_HD bool recheck_incr(const IncrState<W> &st, const Geometry &g, const IncrView<CT, DT> &v) {
  bool ok = true;
  int32_t E = 0;
  for_each_correlation(st, g, [&](int i, int C) {
    E += C * C;
    ok = ok && (v.getC(i) == C);
  });
  ok = ok && (E == st.E);
  for (int a = 0; a < g.D && ok; ++a) ok = ok && (full_delta(st, g, v, a) == v.getD(a));
  return ok;
}

}  // namespace psaw
