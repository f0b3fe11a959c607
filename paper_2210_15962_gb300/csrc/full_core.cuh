// Bit-sliced core of a contiguous self-avoiding walk over the full search
// space of length-L binary sequences (all 2^L of them, any L): the solver the
// paper (arXiv 2210.15962) leaves to future work in Section 5, built from the
// same Eq. 1, Eq. 3 and Algorithm 2.  One CUDA thread owns one walk.
//
// Notation (0-based positions p = 0..L-1; bit b(p) = 1 <-> s_p = -1):
//   flip j (0 <= j < L) negates s_j alone; lags k = 1..L-1 (all parities).
//   A flip changes C_k by -2 u_k, u_k = s_j (s_{j-k} [k <= j] + s_{j+k} [k <= L-1-j]),
//   so Delta_j = sum_k ((C_k - 2 u_k)^2 - C_k^2) = 4 sum u_k^2 - 4 sum u_k C_k.
//   C_k is a sum of L-k terms +-1, so it is odd for L-k odd and even for L-k
//   even.  The signed-digit planes hold the odd numbers C'_k = C_k + [L-k even]
//   (e = (C' + 2^T - 1) / 2, as in walk_core.cuh), and the scan subtracts the
//   offset back: sum u C = sum u C' - sum_{k: L-k even} u_k.
//   The lag windows of flip j are shifts of the one bit array of the sequence:
//   x side b(j-k) (k <= j), y side b(j+k) (k <= L-1-j); they advance one
//   position per flip.
#pragma once
#include "walk_core.cuh"

namespace psaw {

constexpr int kFullLMin = 3;
constexpr int kFullLMax = 256;  // flip index in the low 8 bits of a packed key

// Digit planes per lag-word class W (lags 1..L-1, L <= 32 W + 1):
// |C'_k| <= L <= 2^T - 1.
template <int W>
struct FullPlanesFor {
  static constexpr int value = W == 1 ? 6 : (W == 2 ? 7 : (W <= 4 ? 8 : 9));
};

template <int W, int T>
struct FullState {
  static constexpr int NS = W + 1;  // words of the sequence (L <= 32 W + 1 bits)
  uint32_t bits[NS];                // bit p = b(p); also the walk's visited-table key
  uint32_t ep[T][W];                // digit planes of C'_k, lag k at bit k-1
  int32_t E;
};

// lags k with L-k even (C_k even) as a word pattern: bit i = lag i + 1
LABS_HD uint32_t full_even_lag_mask(int L) { return (L & 1) ? 0x55555555u : 0xAAAAAAAAu; }

// Lag k of the correlations: sh holds the bit array shifted by k - 1 on entry
// and by k on return; C_k = (L - k) - 2 popc(bits ^ sh) over the L - k pairs.
template <int W>
LABS_HD int full_next_correlation(const uint32_t (&bits)[W + 1], uint32_t (&sh)[W + 1], int L, int k) {
  constexpr int NS = W + 1;
#pragma unroll
  for (int w = 0; w < NS; ++w) sh[w] = fshr(sh[w], (w + 1 < NS) ? sh[w + 1] : 0u, 1u);
  const int pairs = L - k;
  int dis = 0;
#pragma unroll
  for (int w = 0; w < NS; ++w) dis += (int)popc32((bits[w] ^ sh[w]) & low_mask_word(pairs, w));
  return pairs - 2 * dis;
}

// P_1 of Eq. 3: L values from the Philox stream (the layout of walk_core.cuh's
// init_walk with L in place of D), then C, E and the digit planes.
template <int W, int T>
LABS_HD void init_full(FullState<W, T> &st, int L, uint64_t seed, uint32_t walk, uint32_t round) {
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
    st.bits[w] = blk[w & 3] & low_mask_word(L, w);
  }
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int w = 0; w < W; ++w) st.ep[t][w] = 0;
  int32_t E = 0;
  uint32_t sh[NS];
#pragma unroll
  for (int w = 0; w < NS; ++w) sh[w] = st.bits[w];
  for (int k = 1; k < L; ++k) {
    const int C = full_next_correlation<W>(st.bits, sh, L, k);
    E += C * C;
    const int Cp = C + (((L - k) & 1) ? 0 : 1);
    const uint32_t e = (uint32_t)((Cp + (1 << T) - 1) >> 1);
#pragma unroll
    for (int t = 0; t < T; ++t) xor_bit(st.ep[t], k - 1, (e >> t) & 1u);
  }
  st.E = E;
}

// Debug recheck: C from XOR + popc against the planes, E against Eq. 1.
template <int W, int T>
LABS_HD bool recheck_full(const FullState<W, T> &st, int L) {
  constexpr int NS = W + 1;
  bool ok = true;
  int32_t E = 0;
  uint32_t sh[NS];
#pragma unroll
  for (int w = 0; w < NS; ++w) sh[w] = st.bits[w];
  for (int k = 1; k < L; ++k) {
    const int C = full_next_correlation<W>(st.bits, sh, L, k);
    E += C * C;
    uint32_t e = 0;
#pragma unroll
    for (int t = 0; t < T; ++t) e |= get_bit(st.ep[t], k - 1) << t;
    const int Cp = C + (((L - k) & 1) ? 0 : 1);
    ok = ok && ((int)(2 * e) - ((1 << T) - 1) == Cp);
  }
  return ok && (E == st.E);
}

// Smallest TP (T-3 <= TP <= T) whose TP-digit form (planes 0..TP-2 and T-1)
// holds every C'_k (the rule of walk_core.cuh's planes_needed over L-1 lags).
template <int W, int T>
LABS_HD int full_planes_needed(const FullState<W, T> &st, int L) {
  uint32_t M[W];
#pragma unroll
  for (int w = 0; w < W; ++w) M[w] = 0xFFFFFFFFu;
  int tp = T;
#pragma unroll
  for (int u = T - 2; u >= T - 4 && u >= 1; --u) {
    bool all = true;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      M[w] &= st.ep[u][w] ^ st.ep[T - 1][w];
      const uint32_t valid = low_mask_word(L - 1, w);
      all = all && ((M[w] & valid) == valid);
    }
    if (!all) break;
    tp = u + 1;
  }
  return tp;
}

// Valid-lag masks of every flip: row j at j * kRowWords holds Vx[0..W-1]
// (lags 1..j), Vy[0..W-1] (lags 1..L-1-j) and the number of lags with L-k
// even that only one side has (|(Vx ^ Vy) & evm|, a term of Qev that depends
// on the flip alone), padded to 16 bytes.
template <int W>
struct FullMaskTable {
  static constexpr int kRowWords = (2 * W + 1 + 3) / 4 * 4;
  static constexpr int kRows = 32 * W + 1;  // >= L
  static constexpr int kWords = kRows * kRowWords;
};

template <int W>
LABS_HD void fill_full_mask_rows(int L, uint32_t *tab, int first, int step) {
  using MT = FullMaskTable<W>;
  const uint32_t evm = full_even_lag_mask(L);
  for (int r = first; r < MT::kRows; r += step) {
    uint32_t *row = tab + (size_t)r * MT::kRowWords;
    for (int k = 0; k < MT::kRowWords; ++k) row[k] = 0u;
    if (r >= L) continue;
    uint32_t c1 = 0;
    for (int w = 0; w < W; ++w) {
      row[w] = low_mask_word(r, w);
      row[W + w] = low_mask_word(L - 1 - r, w);
      c1 += popc32((row[w] ^ row[W + w]) & evm);
    }
    row[2 * W] = c1;
  }
}

template <int W>
LABS_HD void load_full_row(const uint32_t *row, uint32_t (&Vx)[W], uint32_t (&Vy)[W], uint32_t &c1) {
  using MT = FullMaskTable<W>;
  uint32_t r[MT::kRowWords];
#if defined(__CUDA_ARCH__)
#pragma unroll
  for (int k = 0; k < MT::kRowWords / 4; ++k) {
    const uint4 v = reinterpret_cast<const uint4 *>(row)[k];
    r[4 * k] = v.x;
    r[4 * k + 1] = v.y;
    r[4 * k + 2] = v.z;
    r[4 * k + 3] = v.w;
  }
#else
  for (int k = 0; k < MT::kRowWords; ++k) r[k] = row[k];
#endif
#pragma unroll
  for (int w = 0; w < W; ++w) {
    Vx[w] = r[w];
    Vy[w] = r[W + w];
  }
  c1 = r[2 * W];
}

// One flip: the packed key ((Delta + bias) << 8) | j.  B, F: x / y windows
// of the flip, ba = b(j).  With the bits XORed by [s_j = -1] (products
// s_j s_{j-+k}) and the lags split into V1 (one side valid) and V2 (both), as
// in walk_core.cuh's flip_key: S = sum_t 2^t popc(Z_t), M = |M2| (both sides
// equal), Qev = sum over even-C lags of the products' sum,
//   Delta = -8 S + (16 + 8 K1) M + 4 Qev + (4 + 4 K1) n - (8 + 8 K1) n2,
// n = L-1 valid (lag, side) pairs, n2 = |V2| = min(j, L-1-j), K1 = 2^TP - 1.
// Qev = c1 + 2 |M2e| - 2 |V1e & G| - 4 |M2e & G| over the lags with L-k even
// (suffix e), G the product bits, c1 = |V1e| from the mask row.  The two
// G-dependent terms carry S's coefficient; in a two-sided word they join the
// plane sums by one carry-save step, |Z_0| + |A| = |Z_0 ^ A| + 2 |Z_0 & A| with
// A = V1e & G, where Z_0 & A (in V1) and M2e & G (in M2) are disjoint, so
//   S + |A| + 2 |M2e & G| = sum_{t>=1} 2^t |Z_t| + 2 |(Z_0 & A) | (M2e & G)| + |Z_0 ^ A|,
//   Z_0 ^ A = V1 & ((G & ~evm) ^ e_0),  (Z_0 & A) | (M2e & G) = evm & G & ((V1 & ~e_0) | M2),
// one popcount fewer.  The key is then
//   -2048 S' + 256 (16 + 8 K1) M + 1024 Q' + kbase + 1024 c1
// (S' the plane sums with these terms; Q' = 2 |M2e| of the two-sided words
// less 2 |V1e & G| of the one-sided words, where V1 is the valid side) with
//   kbase = 256 ((4 + 4 K1) n - (8 + 8 K1) n2 + bias) + j   (modulo 2^32),
// which moves by a constant per flip on each side of j = L/2; kc = kbase + 1024 c1.
constexpr uint32_t kLutAndNotXor = 0x9A;  // (a & ~b) ^ c
constexpr uint32_t kLutAndNotOr = 0xBA;   // (a & ~b) | c

template <int TP>
LABS_HD uint32_t full_key_base(int j, int L) {
  constexpr uint32_t K1 = (1u << TP) - 1u;
  const int n2 = j < L - 1 - j ? j : L - 1 - j;
  return 256u * ((4u + 4u * K1) * (uint32_t)(L - 1) - (8u + 8u * K1) * (uint32_t)n2 + (uint32_t)kDeltaBias) +
         (uint32_t)j;
}

// NX, NY >= 0 fix at compile time how many leading words have valid x / y
// lags (the caller guarantees NX = ceil(j/32), NY = ceil((L-1-j)/32)); -1
// decides per flip.
template <int W, int T, int TP, int NX = -1, int NY = -1>
LABS_HD uint32_t full_flip_key(const FullState<W, T> &st, const Muls &mu, const uint32_t (&B)[W],
                               const uint32_t (&F)[W], const uint32_t (&Vx)[W], const uint32_t (&Vy)[W],
                               uint32_t ba, int j, int L, uint32_t evm, uint32_t kc) {
  uint32_t acc = 0, mcnt = 0;
  int qev = 0;
  const uint32_t bm = 0u - ba;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    constexpr bool kSkip = W <= kSkipMaxWords;
    const bool xa = NX >= 0 ? (w < NX) : (kSkip ? (j > 32 * w) : true);
    const bool ya = NY >= 0 ? (w < NY) : (kSkip ? (L - 1 - j > 32 * w) : true);
    const uint32_t vx = Vx[w];
    uint32_t v = 0;
    if (xa && ya) {
      const uint32_t vy = Vy[w];
      const uint32_t v1 = vx ^ vy;
      const uint32_t gb = lop3<kLutSelect>(vx, B[w], F[w]) ^ bm;
      const uint32_t m2 = lop3<kLutAndXnor>(vx & vy, B[w], F[w]);
      const uint32_t mall = v1 | m2;
      v = popc32(lop3<kLutAndXor>(m2, gb, st.ep[T - 1][w]));
#pragma unroll
      for (int tt = TP - 1; tt >= 1; --tt) {
        const uint32_t e1 = st.ep[tt < TP - 1 ? tt : T - 1][w];
        const uint32_t e0 = st.ep[tt - 1][w];
        const uint32_t et = lop3<kLutSelect>(v1, e1, e0);
        v = imad(v, mu.two, popc32(lop3<kLutAndXor>(mall, gb, et)));
      }
      // the even-lag terms by the carry-save step above: weight 2 and weight 1
      const uint32_t e0 = st.ep[0][w];
      v = imad(popc32(lop3<kLutAnd3>(evm, gb, lop3<kLutAndNotOr>(v1, e0, m2))), mu.one, v);
      v = imad(v, mu.two, popc32(v1 & lop3<kLutAndNotXor>(gb, evm, e0)));
      mcnt = imad(popc32(m2), mu.one, mcnt);
      qev += 2 * (int)popc32(m2 & evm);
    } else if (xa || ya) {
      const uint32_t m = xa ? vx : Vy[w];
      const uint32_t g = (xa ? B[w] : F[w]) ^ bm;
      v = popc32(lop3<kLutAndXor>(m, g, st.ep[T - 1][w]));
#pragma unroll
      for (int tt = TP - 2; tt >= 0; --tt) v = imad(v, mu.two, popc32(lop3<kLutAndXor>(m, g, st.ep[tt][w])));
      qev -= 2 * (int)popc32(lop3<kLutAnd3>(m, evm, g));
    }
    acc = imad(acc, mu.one, v);
  }
  constexpr uint32_t K1 = (1u << TP) - 1u;
  return imad(acc, (uint32_t)-2048, imad(mcnt, 256u * (16u + 8u * K1), imad((uint32_t)qev, 1024u, kc)));
}

// Flips j0 .. j1-1 (n2 = min(j, L-1-j) on one side of L/2 throughout): packed
// keys into top, skipping j == jprev; the key base advances by `step` per
// flip, the windows B, F and the bit ba by one position.
template <int W, int T, int TP, int K, bool RESCAN, int NX, int NY>
LABS_HD void full_scan_flips(const FullState<W, T> &st, int L, const Muls &mu, const uint32_t *mt, int j0, int j1,
                             uint32_t step, uint32_t evm, int jprev, uint32_t floor, uint32_t (&B)[W],
                             uint32_t (&F)[W], uint32_t &ba, uint32_t (&top)[K]) {
  using MT = FullMaskTable<W>;
  uint32_t Vx[W], Vy[W], c1;
  uint32_t kbase = full_key_base<TP>(j0, L);
  const uint32_t *row = mt + (size_t)j0 * MT::kRowWords;
  for (int j = j0; j < j1; ++j, row += MT::kRowWords, kbase += step) {
    load_full_row<W>(row, Vx, Vy, c1);
    uint32_t x = full_flip_key<W, T, TP, NX, NY>(st, mu, B, F, Vx, Vy, ba, j, L, evm, imad(c1, 1024u, kbase));
    x = (j == jprev || (RESCAN && x < floor)) ? kNone : x;
    top_insert(top, x);
    const uint32_t ba_next = F[0] & 1u;
#pragma unroll
    for (int w = W - 1; w >= 1; --w) B[w] = imadhi(B[w - 1], mu.two, imad(B[w], mu.two, 0u));
    B[0] = imad(B[0], mu.two, ba);
#pragma unroll
    for (int w = 0; w < W; ++w) F[w] = imadhi(F[w], mu.h31, (w + 1 < W) ? imad(F[w + 1], mu.h31, 0u) : 0u);
    ba = ba_next;
  }
}

// One run j0 .. j1-1 whose flips all have nx words with x lags and ny with y
// lags.  Since j + (L-1-j) = L-1 with 32 (W-1) < L-1 <= 32 W, nx + ny is W or
// W+1; those 2W+1 patterns are compiled (P counts them off), any other
// decides per flip.
template <int W, int T, int TP, int K, bool RESCAN, int P = 0>
LABS_HD void full_scan_run(const FullState<W, T> &st, int L, const Muls &mu, const uint32_t *mt, int nx, int ny,
                           int j0, int j1, uint32_t step, uint32_t evm, int jprev, uint32_t floor, uint32_t (&B)[W],
                           uint32_t (&F)[W], uint32_t &ba, uint32_t (&top)[K]) {
  if constexpr (P > 2 * W) {
    full_scan_flips<W, T, TP, K, RESCAN, -1, -1>(st, L, mu, mt, j0, j1, step, evm, jprev, floor, B, F, ba, top);
  } else {
    constexpr int NX = P <= W ? P : P - W;
    constexpr int NY = P <= W ? W - P : 2 * W + 1 - P;
    if (nx == NX && ny == NY)
      full_scan_flips<W, T, TP, K, RESCAN, NX, NY>(st, L, mu, mt, j0, j1, step, evm, jprev, floor, B, F, ba, top);
    else
      full_scan_run<W, T, TP, K, RESCAN, P + 1>(st, L, mu, mt, nx, ny, j0, j1, step, evm, jprev, floor, B, F, ba,
                                                top);
  }
}

// Which lag-word classes scan the full space in pattern runs (chosen by
// measurement): two words, +8% at L=64; four words measured 9% slower at
// L=128, and classes of five words and up keep every word two-sided.
template <int W>
struct FullPatterns {
  static constexpr bool value = W == 2;
};

// Delta_j of all L flips with TP planes; the K smallest packed keys (>= floor
// when RESCAN), skipping j == jprev.  Runs end at L/2, where n2 = min(j,
// L-1-j) turns and the key base's step with it, and, in the classes of
// FullPatterns, where the number of words with x or y lags changes.
template <int W, int T, int TP, int K, bool RESCAN>
LABS_HD void full_eval_tp(const FullState<W, T> &st, int L, const Muls &mu, const uint32_t *mt, int jprev,
                          uint32_t floor, uint32_t (&top)[K]) {
#pragma unroll
  for (int r = 0; r < K; ++r) top[r] = kNone;
  uint32_t F[W], B[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    F[w] = fshr(st.bits[w], st.bits[w + 1], 1u);
    B[w] = 0;
  }
  uint32_t ba = st.bits[0] & 1u;
  const uint32_t evm = full_even_lag_mask(L);
  constexpr uint32_t K1 = (1u << TP) - 1u;
  const int half = L / 2;
  constexpr bool kPatterns = FullPatterns<W>::value && !RESCAN;
  for (int j = 0; j < L;) {
    const uint32_t step = j < half ? 1u - 256u * (8u + 8u * K1) : 1u + 256u * (8u + 8u * K1);
    int j1 = j < half ? half : L;
    if (kPatterns) {
      const int nx = (j + 31) >> 5;
      const int ny = (L - 1 - j + 31) >> 5;
      if (32 * nx + 1 < j1) j1 = 32 * nx + 1;                                 // next change of nx
      if (ny > 0 && L - 1 - 32 * (ny - 1) < j1) j1 = L - 1 - 32 * (ny - 1);  // ... or of ny
      full_scan_run<W, T, TP, K, RESCAN>(st, L, mu, mt, nx, ny, j, j1, step, evm, jprev, floor, B, F, ba, top);
    } else {
      full_scan_flips<W, T, TP, K, RESCAN, -1, -1>(st, L, mu, mt, j, j1, step, evm, jprev, floor, B, F, ba, top);
    }
    j = j1;
  }
}

template <int W, int T, int K>
LABS_HD void full_eval(const FullState<W, T> &st, int L, const Muls &mu, const uint32_t *mt, int tp, int jprev,
                       uint32_t floor, uint32_t (&top)[K]) {
  constexpr int T3 = T - 3 >= 2 ? T - 3 : 2;
  if (floor == 0) {
    if (tp >= T) full_eval_tp<W, T, T, K, false>(st, L, mu, mt, jprev, 0u, top);
    else if (tp == T - 1) full_eval_tp<W, T, T - 1, K, false>(st, L, mu, mt, jprev, 0u, top);
    else if (tp == T - 2) full_eval_tp<W, T, T - 2, K, false>(st, L, mu, mt, jprev, 0u, top);
    else full_eval_tp<W, T, T3, K, false>(st, L, mu, mt, jprev, 0u, top);
  } else {
    full_eval_tp<W, T, T, K, true>(st, L, mu, mt, jprev, floor, top);
  }
}

// Move to the neighbour of flip j: C_k -= 2 u_k on the planes (e += -u_k by a
// bit-sliced add), E += delta, and flip b(j).
template <int W, int T>
LABS_HD void apply_full(FullState<W, T> &st, int L, int j, int delta) {
  constexpr int NS = W + 1;
  const uint32_t ba = get_bit(st.bits, j);
  const uint32_t bm = 0u - ba;
  // Y window: bits j+1 ..; X window: bits j-1, j-2, .. via a full bit reversal
  uint32_t F[W], R[NS], X[W];
  shr_dyn(F, st.bits, j + 1);
#pragma unroll
  for (int w = 0; w < NS; ++w) R[w] = brev32(st.bits[NS - 1 - w]);
  shr_dyn(X, R, 32 * NS - j);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t vx = low_mask_word(j, w);
    const uint32_t vy = low_mask_word(L - 1 - j, w);
    const uint32_t Xw = X[w] ^ bm, Yw = F[w] ^ bm;  // product bits (1 <-> s_j s_{j-+k} = -1)
    // g = -product in {-1, 0, 1} (0 where the side is not valid): bit 0 = valid, sign = valid & ~product
    const uint32_t x0 = vx, xs = vx & ~Xw;
    const uint32_t y0 = vy, ys = vy & ~Yw;
    // d = g_x + g_y = -u in [-2, 2], three-bit two's complement
    const uint32_t d0 = x0 ^ y0;
    const uint32_t c1 = x0 & y0;
    const uint32_t d1 = xs ^ ys ^ c1;
    const uint32_t c2 = (xs & ys) | (c1 & (xs ^ ys));
    const uint32_t d2 = xs ^ ys ^ c2;
    // e += d over T planes (addend planes d0, d1, d2, d2, ...)
    uint32_t carry = 0;
#pragma unroll
    for (int tt = 0; tt < T; ++tt) {
      const uint32_t add = tt == 0 ? d0 : (tt == 1 ? d1 : d2);
      const uint32_t e = st.ep[tt][w];
      st.ep[tt][w] = lop3<kLutXor3>(e, add, carry);
      carry = lop3<kLutMajority>(e, add, carry);
    }
  }
  st.E += delta;
  xor_bit(st.bits, j, 1u);
}

}  // namespace psaw
