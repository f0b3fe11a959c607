// Bit-sliced core of one contiguous self-avoiding walk over skew-symmetric
// binary sequences (Bošković, Herzog, Brest, arXiv 2210.15962, Eq. 1-3 and
// Algorithm 2).  One CUDA thread owns one walk; every array below lives in
// that thread's registers (all indices are compile-time after unrolling).
//
// Notation (0-based positions a = 0..L-1; the paper's s_{a+1}):
//   D = (L+1)/2 free positions 0..D-1, centre c = D-1, m = (L-1)/2 even lags
//   k = 2i (i = 1..m).  Bit b(a) = 1 <-> s_a = -1.  Flip j negates position
//   a = j and its mirror a' = L-1-j (Eq. 2), which is a itself when j = c.
//
// Facts used (each follows from Eq. 1 and Eq. 2):
//   * C_k = 0 for odd k, and for even k the flip changes
//       C_{2i} by -4 u_i,  u_i = s_a (s_{a-2i} [a-2i >= 0] + s_{a+2i} [a+2i <= L-1, a+2i != a'])
//     (only the s_{a-2i} term for the centre), so the neighbour's energy change is
//       Delta_j = sum_i (-4u_i)(2 C_{2i} - 4u_i) = 16 sum_i u_i^2 - 8 sum_i u_i C_{2i};
//   * positions a and a +- 2i have the same parity, so each parity class of
//     positions is kept as its own bit array ("cls"); the windows of bits at
//     a-2i and a+2i over all lags i are plain shifts of that array;
//   * every C_{2i} is odd (a sum of L-2i terms +-1), so it has a unique
//     T-digit signed-binary form C = sum_t 2^t d_t with d_t in {-1,+1};
//     the digit bits e_t = (d_t+1)/2 are the bits of e = (C + 2^T - 1)/2, held
//     as T bit planes over the lags ("ep").  With x'_i = s_a s_{a-2i} = 1-2X_i,
//       sum_{i in V} x'_i C_{2i} = 2 sum_t 2^t popc(V & (X ^ e_t)) - (2^T-1)|V|,
//     so a neighbour costs, per 32 lags and digit plane, one select, one
//     masked XOR and one population count (both sides at once, see flip_key).
#pragma once
#include <stddef.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define LABS_HD __host__ __device__ __forceinline__
#else
#define LABS_HD inline
#endif

namespace psaw {

// ---------------------------------------------------------------- limits
constexpr int kLMin = 5;
constexpr int kLMax = 511;        // D <= 256 free bits, m <= 255 lags
constexpr int kMaxWords = 8;      // 32-bit words of lags (m <= 32 * kMaxWords)
constexpr int kKeyWords = 9;      // 32-bit words of a key (D bits + occupancy flag)
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kDeltaBias = 1 << 22;  // |Delta| < 2^21 for L <= 511
constexpr int kSkipMaxWords = 4;     // classes up to this many lag words skip empty word sides

LABS_HD uint32_t popc32(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return (uint32_t)__popc(x);
#else
  return (uint32_t)__builtin_popcount(x);
#endif
}

// low 32 bits of (hi:lo) >> s, 0 <= s <= 31
LABS_HD uint32_t fshr(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, s);
#else
  s &= 31u;
  return s ? ((lo >> s) | (hi << (32u - s))) : lo;
#endif
}

LABS_HD uint32_t brev32(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __brev(x);
#else
  x = ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
  x = ((x >> 2) & 0x33333333u) | ((x & 0x33333333u) << 2);
  x = ((x >> 4) & 0x0F0F0F0Fu) | ((x & 0x0F0F0F0Fu) << 4);
  x = ((x >> 8) & 0x00FF00FFu) | ((x & 0x00FF00FFu) << 8);
  return (x >> 16) | (x << 16);
#endif
}

LABS_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// word w of the mask whose low n bits are set (n may be <= 0)
LABS_HD uint32_t low_mask_word(int n, int w) {
  const int s = n - 32 * w;
  return s <= 0 ? 0u : (s >= 32 ? 0xFFFFFFFFu : ((1u << s) - 1u));
}

// Dynamic-position access to small register arrays.  Each word is selected
// with an AND mask rather than an index so that the array stays in registers.
LABS_HD uint32_t sel_mask(bool b) { return 0u - (uint32_t)b; }

// bit `pos` of a register array
template <int N>
LABS_HD uint32_t get_bit(const uint32_t (&a)[N], int pos) {
  uint32_t w = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) w |= a[i] & sel_mask((pos >> 5) == i);
  return (w >> (pos & 31)) & 1u;
}

template <int N>
LABS_HD void xor_bit(uint32_t (&a)[N], int pos, uint32_t v) {
  const uint32_t b = v << (pos & 31);
#pragma unroll
  for (int i = 0; i < N; ++i) a[i] ^= b & sel_mask((pos >> 5) == i);
}

// out = bits [s, s + 32*NO) of a (zero past the end), s >= 0 dynamic
template <int NO, int NI>
LABS_HD void shr_dyn(uint32_t (&out)[NO], const uint32_t (&a)[NI], int s) {
  const int ws = s >> 5;
  const uint32_t bs = (uint32_t)(s & 31);
#pragma unroll
  for (int w = 0; w < NO; ++w) {
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      lo |= a[i] & sel_mask(i == w + ws);
      hi |= a[i] & sel_mask(i == w + ws + 1);
    }
    out[w] = fshr(lo, hi, bs);
  }
}

// ------------------------------------------------- Philox4x32-10 generator
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of
//   (x0,x1,x2,x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))
// with the key advanced by the Weyl increments after each round.
LABS_HD void philox4x32_10(uint32_t (&x)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * x[0], hi0 = mulhi32(0xD2511F53u, x[0]);
    const uint32_t lo1 = 0xCD9E8D57u * x[2], hi1 = mulhi32(0xCD9E8D57u, x[2]);
    const uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// ----------------------------------------------------------- problem shape
struct Geometry {
  int L, D, c, m;
  int N[2];      // sizes of the two parity classes (D and D-1)
  int nfree[2];  // free positions (a < D) in each class
  int T;         // digit planes
};

LABS_HD Geometry make_geometry(int L, int T) {
  Geometry g;
  g.L = L;
  g.D = (L + 1) / 2;
  g.c = g.D - 1;
  g.m = (L - 1) / 2;
  g.N[0] = g.D;
  g.N[1] = g.D - 1;
  g.nfree[0] = (g.D + 1) / 2;
  g.nfree[1] = g.D / 2;
  g.T = T;
  return g;
}

// smallest T with 2^T - 1 >= L - 2 (the largest |C_{2i}|)
LABS_HD int digits_for(int L) {
  int T = 1;
  while ((1 << T) < L - 1) ++T;
  return T;
}

// ------------------------------------------------------- valid-lag masks
// The lags a flip's windows cover depend only on its parity class q and class
// index t (a = 2t + q), not on the sequence: x side lags 1..t, y side lags
// 1..N_q-1-t without the lag c - a of the flip's own mirror (empty for the
// centre).  They are tabulated once per L: row (q, t) at
// (q * kMaskRows<W> + t) * kMaskRowWords<W> holds Vx[0..W-1] then Vye[0..W-1],
// padded to 16 bytes.
template <int W>
struct MaskTable {
  static constexpr int kRowWords = (2 * W + 3) / 4 * 4;
  static constexpr int kRows = 16 * W + 1;  // >= nfree[0] = (D + 1) / 2 for m <= 32 W
  static constexpr int kWords = 2 * kRows * kRowWords;
};

// Rows first, first + step, ... of the table for geometry g (rows past a
// class's last flip are zero).
template <int W>
LABS_HD void fill_mask_rows(const Geometry &g, uint32_t *tab, int first, int step) {
  using MT = MaskTable<W>;
  for (int r = first; r < 2 * MT::kRows; r += step) {
    const int q = r >= MT::kRows ? 1 : 0;
    const int t = r - q * MT::kRows;
    uint32_t *row = tab + (size_t)r * MT::kRowWords;
    for (int k = 0; k < MT::kRowWords; ++k) row[k] = 0u;
    if (t >= g.nfree[q]) continue;
    const int a = 2 * t + q;
    const bool centre = (a == g.c);
    const int i0 = g.c - a;
    for (int w = 0; w < W; ++w) {
      row[w] = low_mask_word(t, w);
      uint32_t vy = centre ? 0u : low_mask_word(g.N[q] - 1 - t, w);
      if (!centre && ((i0 - 1) >> 5) == w) vy &= ~(1u << ((i0 - 1) & 31));
      row[W + w] = vy;
    }
  }
}

// Row (q, t) of the table into registers (16-byte loads on the device).
template <int W>
LABS_HD void load_mask_row(const uint32_t *row, uint32_t (&Vx)[W], uint32_t (&Vye)[W]) {
  using MT = MaskTable<W>;
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
    Vye[w] = r[W + w];
  }
}

// ------------------------------------------------------------- walk state
// W: 32-bit words of lags; T: digit planes; NS = W + 1 words per class.
template <int W, int T>
struct WalkState {
  static constexpr int NS = W + 1;
  uint32_t cls[2][NS];  // cls[q] bit t = b(2t + q)
  uint32_t ep[T][W];    // ep[t] bit (i-1) = bit t of e_i = (C_{2i} + 2^T - 1) / 2
  uint32_t key[NS];     // key bit j = b(j), j < D (the free half identifies a skew pivot)
  int32_t E;            // energy of the current pivot, Eq. 1
};

// C_{2i} from the class arrays with XOR + popc on packed words: the pairs
// (a, a+2i) inside class q are (t, t+i), t = 0..N_q-1-i, and
// C = (#pairs) - 2 (#disagreeing pairs).  Called for i = 1, 2, ... in order;
// sh[q] holds cls[q] >> (i-1) on entry and cls[q] >> i on return.
template <int W, int T>
LABS_HD int next_even_correlation(const WalkState<W, T> &st, const Geometry &g, uint32_t (&sh)[2][W + 1], int i) {
  constexpr int NS = W + 1;
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
  return C;
}

// P_1 of Eq. 3: free bit j = bit (j%32) of word (j/32)%4 of
// Philox(counter = (walk, round, j/128, 0), key = seed), 1 <-> -1; then
// Eq. 2 fills the second half, and Eq. 1 gives C and E.
template <int W, int T>
LABS_HD void init_walk(WalkState<W, T> &st, const Geometry &g, uint64_t seed, uint32_t walk, uint32_t round) {
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
      const int i = a - g.c;                       // s_{c+i} = (-1)^i s_{c-i}
      b = get_bit(st.key, g.c - i) ^ (uint32_t)(i & 1);
    }
    if (a & 1) xor_bit(st.cls[1], a >> 1, b);
    else xor_bit(st.cls[0], a >> 1, b);
  }
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int w = 0; w < W; ++w) st.ep[t][w] = 0;
  int32_t E = 0;
  uint32_t sh[2][NS];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int w = 0; w < NS; ++w) sh[q][w] = st.cls[q][w];
  for (int i = 1; i <= g.m; ++i) {
    const int C = next_even_correlation(st, g, sh, i);
    E += C * C;
    const uint32_t e = (uint32_t)((C + (1 << T) - 1) >> 1);
#pragma unroll
    for (int t = 0; t < T; ++t) xor_bit(st.ep[t], i - 1, (e >> t) & 1u);
  }
  st.E = E;
}

// Full recheck (debug): recompute every C_{2i} with XOR + popc and E from
// Eq. 1 and compare with the digit planes and the running E.
template <int W, int T>
LABS_HD bool recheck_walk(const WalkState<W, T> &st, const Geometry &g) {
  constexpr int NS = W + 1;
  bool ok = true;
  int32_t E = 0;
  uint32_t sh[2][NS];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int w = 0; w < NS; ++w) sh[q][w] = st.cls[q][w];
  for (int i = 1; i <= g.m; ++i) {
    const int C = next_even_correlation(st, g, sh, i);
    E += C * C;
    uint32_t e = 0;
#pragma unroll
    for (int t = 0; t < T; ++t) e |= get_bit(st.ep[t], i - 1) << t;
    ok = ok && ((int)(2 * e) - ((1 << T) - 1) == C);
  }
  return ok && (E == st.E);
}

// insert x into the ascending list top[0..K-1] (the largest drops off)
template <int K>
LABS_HD void top_insert(uint32_t (&top)[K], uint32_t x) {
#pragma unroll
  for (int r = 0; r < K; ++r) {
    const uint32_t lo = top[r] < x ? top[r] : x;
    x = top[r] < x ? x : top[r];
    top[r] = lo;
  }
}

// Integer multiply-adds with a multiplier that is a run-time value, so that
// they execute on the FMA pipe as IMAD (the ALU pipe carries the bit logic).
// With m = 2, 2^31 or 2^30 they implement shifts: umulhi(x, 2^31) = x >> 1,
// x * 2^31 = (x & 1) << 31, umulhi(x, 2) = x >> 31.
struct Muls {
  uint32_t one, two, four, h31, h30;
};

LABS_HD uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
#else
  return a * b + c;
#endif
}

LABS_HD uint32_t imadhi(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
  uint32_t d;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
#else
  return (uint32_t)(((uint64_t)a * b) >> 32) + c;
#endif
}

// Three-input bit function by its lookup table (the PTX lop3 encoding: LUT =
// f(0xF0, 0xCC, 0xAA) for f of (a, b, c)), one LOP3 on the device.
template <uint32_t LUT>
LABS_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
#else
  uint32_t r = 0;
  for (int i = 0; i < 8; ++i)
    if ((LUT >> i) & 1u) r |= ((i & 4) ? a : ~a) & ((i & 2) ? b : ~b) & ((i & 1) ? c : ~c);
  return r;
#endif
}
constexpr uint32_t kLutAndXor = 0x60;     // a & (b ^ c)
constexpr uint32_t kLutSelect = 0xCA;     // a ? b : c, bitwise
constexpr uint32_t kLutAndXnor = 0x90;    // a & ~(b ^ c)
constexpr uint32_t kLutXor3 = 0x96;       // a ^ b ^ c
constexpr uint32_t kLutMajority = 0xE8;   // at least two of a, b, c
constexpr uint32_t kLutAnd3 = 0x80;       // a & b & c

// Smallest number of digit planes TP (T-3 <= TP <= T) that represents every
// current C_{2i}: |C| <= 2^TP - 1 holds iff the digit bits TP-1 .. T-2 of
// every e_i differ from its top bit T-1.  The TP-digit form of C then uses
// planes 0 .. TP-2 and plane T-1 (as digit TP-1); any TP at or above this
// minimum gives the same exact sums.
template <int W, int T>
LABS_HD int planes_needed(const WalkState<W, T> &st, const Geometry &g) {
  uint32_t M[W];
#pragma unroll
  for (int w = 0; w < W; ++w) M[w] = 0xFFFFFFFFu;
  int tp = T;
#pragma unroll
  for (int u = T - 2; u >= T - 4 && u >= 1; --u) {  // tp = u + 1 >= T - 3
    bool all = true;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      M[w] &= st.ep[u][w] ^ st.ep[T - 1][w];
      const uint32_t valid = low_mask_word(g.m, w);
      all = all && ((M[w] & valid) == valid);
    }
    if (!all) break;
    tp = u + 1;
  }
  return tp;
}

// One flip of the neighbourhood scan.  B, F: bits at a-2i and a+2i of the
// flip's class (lags i = 1.. on bits 0..); Vx, Vye: valid lags of each side
// (Vye without the flip's own mirror pair); ba: the bit of position a.
// Returns the packed key ((Delta + bias) << 8) | a.
//   Q0 = sum_i (s_{a-2i} [i in Vx] + s_{a+2i} [i in Vye]) C_{2i}
//      = 2 P - (2^TP - 1)(|Vx| + |Vye|),  P = sum_t 2^t popc over both sides of (V & (window ^ e_t)),
//   Q = s_a Q0,  R = |Vx| + |Vye| + 2 |Vx & Vye| - 4 popc(Vx & Vye & (B ^ F)),
//   Delta = 16 R - 8 Q.
// The lags split into V1 = Vx ^ Vye (one side valid, bit G of that side) and
// V2 = Vx & Vye.  A lag of V2 whose two bits differ adds 2^TP - 1 to P
// whatever C is; one whose bits agree (M2 = V2 & ~(B ^ F)) adds twice its
// one-sided term, i.e. its term one digit higher.  V1 and M2 are disjoint, so
//   P = sum_{t=0..TP} 2^t popc(Z_t) + (2^TP - 1)(|V2| - |M2|),
//   Z_t = (V1 & (G ^ e_t)) | (M2 & (G ^ e_{t-1})) = (V1 | M2) & (G ^ (V1 ? e_t : e_{t-1})),
// two LOP3 and one POPC per plane and word.  The bits enter XORed with
// [s_a = -1], so that they stand for the products s_a s_{a-+2i}: with
// S = sum_t 2^t popc(Z_t) over the words, M = sum of |M2| and |V2| = nxy,
//   Delta = -16 S + 16 (K1 + 4) M + (16 + 8 K1) n - (32 + 16 K1) nxy,  K1 = 2^TP - 1,
// the same for both signs of s_a (R does not depend on it, and Q = 2 P - K1 n
// with P taken over the products).
// How the sign s_a enters, per lag-word class (chosen by measurement): folded
// into the bits (one XOR per active word) or by coefficients selected by s_a
// (three IMAD per flip).  Classes with few active words gain from the fold
// (L=121 +1.3%, L=301 +8%); at 4 and 6..8 words the selected form measured
// 3-7% faster.
template <int W>
struct FoldSign {
  static constexpr bool value = W <= 3 || W == 5;
};

// Words of a class that can hold x lags: a scanned flip has t <= (D-1)/2 = m/2
// <= 16 W, so its x lags i <= t lie in the first ceil(W/2) words.
template <int W>
constexpr int x_words() {
  return (W + 1) / 2;
}

// The part of a flip's key that the bit counts do not enter.  The key is
// 256 (Delta + bias) + a; with Delta as below and n = |Vx| + |Vye|,
// nxy = |Vx & Vye| it is
//   key = -4096 S + 4096 (K1 + 4) M + kbase                          (s_a folded into the bits)
//   key = 256 sig S + 256 mul M + kbase + [s_a = -1] kdiff           (coefficients selected by s_a)
//   kbase = 256 (bias + (16 + 8 K1) n - (32 + 16 K1) nxy) + a,  kdiff = 256 (32 K1 nxy - 16 K1 n),
// all modulo 2^32 like the key.  Along a run of flips n is fixed and a, nxy
// grow by 2 and 1 per flip (while the pair lag stays on one side of t), so
// both advance by a constant step.
template <int TP>
LABS_HD uint32_t key_base(int a, int n, int nxy) {
  constexpr uint32_t K1 = (1u << TP) - 1u;
  return 256u * ((uint32_t)kDeltaBias + (16u + 8u * K1) * (uint32_t)n - (32u + 16u * K1) * (uint32_t)nxy) +
         (uint32_t)a;
}
template <int TP>
LABS_HD uint32_t key_diff(int n, int nxy) {
  constexpr uint32_t K1 = (1u << TP) - 1u;
  return 256u * (32u * K1 * (uint32_t)nxy - 16u * K1 * (uint32_t)n);
}

// How the scan forms key_base / key_diff, per lag-word class (chosen by
// measurement): advanced by a constant step along runs that end where the
// pair lag changes side, or computed from a and nxy at every flip.  The
// stepped form measured 3-20% faster at 2 and 4..8 words, 5-6% slower at 1
// and 3 words.
template <int W>
struct SteppedKey {
  static constexpr bool value = W != 1 && W != 3;
};

// NX, NY >= 0 fix at compile time how many leading words have valid x / y
// lags (the caller guarantees NX = ceil(t/32), NY = ceil((Nq-1-t)/32));
// -1 decides per flip.  ALL_WORDS evaluates every word that can hold lags
// on the two-sided path without testing which sides are empty (an empty
// side's zero mask makes its terms vanish), for callers whose lanes hold
// different flips.  kbase, kdiff: the flip's key_base / key_diff.
template <int W, int T, int TP, bool CENTRE, int NX = -1, int NY = -1, bool ALL_WORDS = false>
LABS_HD uint32_t flip_key(const WalkState<W, T> &st, const Muls &mu, const uint32_t (&B)[W], const uint32_t (&F)[W],
                          const uint32_t (&Vx)[W], const uint32_t (&Vye)[W], uint32_t ba, uint32_t kbase,
                          uint32_t kdiff, int t, int Nq) {
  constexpr bool kFold = FoldSign<W>::value;
  uint32_t acc = 0, mcnt = 0;
  const uint32_t bm = kFold ? 0u - ba : 0u;  // all ones where s_a = -1 (folded form)
#pragma unroll
  for (int w = 0; w < W; ++w) {
    // which sides have valid lags in this word (the same for every lane of the warp):
    // x lags i <= t, y lags i <= Nq-1-t.  Wide classes keep every word on the
    // two-sided path: with few resident warps they rely on the compiler
    // interleaving the words' independent chains.
    constexpr bool kSkip = W <= kSkipMaxWords && !ALL_WORDS;
    const bool xa = w < x_words<W>() && (NX >= 0 ? (w < NX) : (kSkip ? (t > 32 * w) : true));
    const bool ya = CENTRE ? false : (NY >= 0 ? (w < NY) : (kSkip ? (Nq - 1 - t > 32 * w) : true));
    const uint32_t vx = Vx[w];
    uint32_t v = 0;
    // digits from the top down, each count entering the Horner sum sum_t 2^t popc(Z_t) at once
    if (xa && ya) {
      const uint32_t vy = Vye[w];
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
      v = imad(v, mu.two, popc32(lop3<kLutAndXor>(v1, gb, st.ep[0][w])));
      mcnt = imad(popc32(m2), mu.one, mcnt);
    } else if (xa || ya) {
      const uint32_t m = xa ? vx : Vye[w];
      const uint32_t g = (xa ? B[w] : F[w]) ^ bm;
      v = popc32(lop3<kLutAndXor>(m, g, st.ep[T - 1][w]));
#pragma unroll
      for (int tt = TP - 2; tt >= 0; --tt) v = imad(v, mu.two, popc32(lop3<kLutAndXor>(m, g, st.ep[tt][w])));
    }
    acc = imad(acc, mu.one, v);
  }
  constexpr uint32_t K1 = (1u << TP) - 1u;
  if constexpr (kFold) {
    return imad(acc, (uint32_t)-4096, imad(mcnt, 4096u * (K1 + 4u), kbase));
  } else {
    // bits not folded: S and M are taken over the window bits themselves, and
    //   s_a = +1: Delta = -16 S + 16 (K1 + 4) M + 8 K1 n + 16 n + 32 nxy - 16 (K1 + 4) nxy
    //   s_a = -1: Delta = +16 S - 16 (K1 - 4) M - 8 K1 n + 16 n - 32 nxy + 16 K1 nxy
    // (the s_a = +1 constant is kbase's, the difference kdiff's)
    const uint32_t sig = imad(ba, 8192u, (uint32_t)-4096);
    const uint32_t mul = imad(ba, 0u - 8192u * K1, 4096u * (K1 + 4u));
    const uint32_t kap = imad(ba, kdiff, kbase);
    return imad(acc, sig, imad(mcnt, mul, kap));
  }
}

// Flips t0 .. t1-1 of class q (none of them the centre; with SteppedKey, the
// pair lag c - a on one side of t throughout: t >= tpair for all of them or
// for none): packed keys into top, skipping t == tprev; windows B, F and the
// bit ba of position a advanced one lag per flip.
template <int W, int T, int TP, int K, bool RESCAN, int NX, int NY, int U = 1>
LABS_HD void scan_flips(const WalkState<W, T> &st, const Geometry &g, const Muls &mu, const uint32_t *rows, int q,
                        int t0, int t1, int tprev, int tpair, uint32_t floor, uint32_t (&B)[W], uint32_t (&F)[W],
                        uint32_t &ba, uint32_t (&top)[K]) {
  using MT = MaskTable<W>;
  constexpr uint32_t K1 = (1u << TP) - 1u;
  const int Nq = g.D - q;  // N_q without indexing g.N
  const int n = Nq - 2;    // |Vx| + |Vye| for every non-centre flip
  // |Vx & Vye| = min(t, Nq-1-t) = t in the scan (t <= (Nq-1)/2), less the
  // pair lag c - a if it is <= t, i.e. if t >= tpair
  const int nxy0 = t0 - (t0 >= tpair ? 1 : 0);
  uint32_t kbase = key_base<TP>(2 * t0 + q, n, nxy0);
  uint32_t kdiff = key_diff<TP>(n, nxy0);
  const uint32_t *row = rows + (size_t)t0 * MT::kRowWords;
  auto one_flip = [&](int t) {
    uint32_t Vx[W], Vye[W];
    load_mask_row<W>(row, Vx, Vye);
    if constexpr (!SteppedKey<W>::value) {
      const int nxy = t - (t >= tpair ? 1 : 0);
      kbase = key_base<TP>(2 * t + q, n, nxy);
      kdiff = key_diff<TP>(n, nxy);
    }
    uint32_t x = flip_key<W, T, TP, false, NX, NY>(st, mu, B, F, Vx, Vye, ba, kbase, kdiff, t, Nq);
    x = (t == tprev || (RESCAN && x < floor)) ? kNone : x;
    top_insert(top, x);
    kbase += 2u - 256u * (32u + 16u * K1);  // a += 2, nxy += 1
    kdiff += 256u * 32u * K1;
    // advance the windows by one lag (shifts as IMAD on the FMA pipe); the x
    // window only over the words that can hold x lags
    const uint32_t ba_next = F[0] & 1u;
#pragma unroll
    for (int w = x_words<W>() - 1; w >= 1; --w) B[w] = imadhi(B[w - 1], mu.two, imad(B[w], mu.two, 0u));
    B[0] = imad(B[0], mu.two, ba);
#pragma unroll
    for (int w = 0; w < W; ++w) F[w] = imadhi(F[w], mu.h31, (w + 1 < W) ? imad(F[w + 1], mu.h31, 0u) : 0u);
    ba = ba_next;
  };
  if constexpr (U == 1) {
    for (int t = t0; t < t1; ++t, row += MT::kRowWords) one_flip(t);
  } else {
    // U > 1 unrolls the flip loop, giving the scheduler U flips' independent
    // popcount chains at once (a launch-shape knob of the batch autotuner)
#pragma unroll(U)
    for (int t = t0; t < t1; ++t, row += MT::kRowWords) one_flip(t);
  }
}

// Classes of kPatternMinWords .. PMAX lag words (PMAX a template parameter of
// the scan, chosen per kernel) scan in runs of flips with a fixed pattern of
// active word sides, each run through a loop compiled for it (one-word classes
// have too few flips per run to gain).
constexpr int kPatternMinWords = 2;

// One run t0 .. t1-1 whose flips all have nx words with x lags and ny with y
// lags.  The patterns compiled are nx = 0 .. ceil(W/2) (t <= 16 W) and
// ny = max(1, W/2) .. W (the y side keeps at least half the class); any other
// pattern decides per flip.
template <int W, int T, int TP, int K, bool RESCAN, int NX = 0, int NY = (W / 2 > 1 ? W / 2 : 1), int U = 1>
LABS_HD void scan_run(const WalkState<W, T> &st, const Geometry &g, const Muls &mu, const uint32_t *rows, int q,
                      int nx, int ny, int t0, int t1, int tprev, int tpair, uint32_t floor, uint32_t (&B)[W],
                      uint32_t (&F)[W], uint32_t &ba, uint32_t (&top)[K]) {
  if constexpr (NX > (W + 1) / 2) {
    scan_flips<W, T, TP, K, RESCAN, -1, -1, U>(st, g, mu, rows, q, t0, t1, tprev, tpair, floor, B, F, ba, top);
  } else if constexpr (NY > W) {
    scan_run<W, T, TP, K, RESCAN, NX + 1, (W / 2 > 1 ? W / 2 : 1), U>(st, g, mu, rows, q, nx, ny, t0, t1, tprev, tpair,
                                                                   floor, B, F, ba, top);
  } else {
    if (nx == NX && ny == NY)
      scan_flips<W, T, TP, K, RESCAN, NX, NY, U>(st, g, mu, rows, q, t0, t1, tprev, tpair, floor, B, F, ba, top);
    else
      scan_run<W, T, TP, K, RESCAN, NX, NY + 1, U>(st, g, mu, rows, q, nx, ny, t0, t1, tprev, tpair, floor, B, F, ba,
                                                top);
  }
}

// Delta_j of every flip j of the pivot (Algorithm 2, the neighbourhood evaluation)
// with TP digit planes, and the K smallest packed keys (>= floor when RESCAN),
// skipping j == jprev (the previous pivot, always visited).  Flips are scanned
// class by class; the bit windows advance by one lag per flip and the valid-lag
// masks come from the table mt (MaskTable<W>, filled for this geometry).  In
// narrow classes the flips of a class split into runs where the number of
// words with x lags, ceil(t/32), and with y lags, ceil((Nq-1-t)/32), is fixed.
template <int W, int T, int TP, int K, bool RESCAN, int PMAX, int U = 1>
LABS_HD void eval_neighbours_tp(const WalkState<W, T> &st, const Geometry &g, const Muls &mu, const uint32_t *mt,
                                int jprev, uint32_t floor, uint32_t (&top)[K]) {
  using MT = MaskTable<W>;
#pragma unroll
  for (int r = 0; r < K; ++r) top[r] = kNone;
  // one pass per parity class, unrolled only for one-word classes (wider
  // classes' loops are large and share the instruction caches); the class
  // array is selected without dynamic indexing
#pragma unroll(W == 1 ? 2 : 1)
  for (int q = 0; q < 2; ++q) {
    const int Nq = g.D - q;
    const uint32_t *rows = mt + (size_t)q * MT::kRows * MT::kRowWords;
    const uint32_t mq = sel_mask(q != 0);
    uint32_t F[W], B[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c0 = (st.cls[1][w] & mq) | (st.cls[0][w] & ~mq);
      const uint32_t c1 = (st.cls[1][w + 1] & mq) | (st.cls[0][w + 1] & ~mq);
      F[w] = fshr(c0, c1, 1u);
      B[w] = 0;
    }
    uint32_t ba = ((st.cls[1][0] & mq) | (st.cls[0][0] & ~mq)) & 1u;
    const bool has_centre = (g.c & 1) == q;
    const int nloop = (q ? g.D / 2 : (g.D + 1) / 2) - (has_centre ? 1 : 0);
    // the previous pivot's flip index in this class (-1: none), and the first
    // t whose pair lag c - a = c - 2t - q is <= t
    const int tprev = (jprev >= 0 && (jprev & 1) == q) ? (jprev >> 1) : -1;
    const int tpair = (g.c - q + 2) / 3;
    if (W >= kPatternMinWords && W <= PMAX && !RESCAN) {
      for (int t = 0; t < nloop;) {
        const int nx = (t + 31) >> 5;
        const int ly = Nq - 1 - t;
        const int ny = ly > 0 ? (ly + 31) >> 5 : 0;
        int t1 = 32 * nx + 1;                                             // next change of nx
        if (ny > 0 && Nq - 1 - 32 * (ny - 1) < t1) t1 = Nq - 1 - 32 * (ny - 1);  // ... or of ny
        if (SteppedKey<W>::value && t < tpair && tpair < t1) t1 = tpair;  // ... or of the pair lag's side
        if (t1 > nloop) t1 = nloop;
        scan_run<W, T, TP, K, RESCAN, 0, (W / 2 > 1 ? W / 2 : 1), U>(st, g, mu, rows, q, nx, ny, t, t1, tprev, tpair,
                                                                    floor, B, F, ba, top);
        t = t1;
      }
    } else {
      for (int t = 0; t < nloop;) {  // with SteppedKey two runs, split where the pair lag changes side
        const int t1 = (SteppedKey<W>::value && t < tpair && tpair < nloop) ? tpair : nloop;
        scan_flips<W, T, TP, K, RESCAN, -1, -1, U>(st, g, mu, rows, q, t, t1, tprev, tpair, floor, B, F, ba, top);
        t = t1;
      }
    }
    if (has_centre) {
      const int t = nloop, a = g.c;
      uint32_t Vx[W], Vye[W];
      load_mask_row<W>(rows + (size_t)t * MT::kRowWords, Vx, Vye);
      // the centre has n = |Vx| = t and no y side (nxy = 0)
      uint32_t x = flip_key<W, T, TP, true>(st, mu, B, F, Vx, Vye, ba, key_base<TP>(a, t, 0), key_diff<TP>(t, 0), t,
                                            Nq);
      x = (a == jprev || (RESCAN && x < floor)) ? kNone : x;
      top_insert(top, x);
    }
  }
}

// Dispatch on the plane count (the caller may pass any tp >= planes_needed);
// floor > 0 selects the rescan variant (candidates at or above floor only).
template <int W, int T, int K, bool RESCAN, int PMAX, int U = 1>
LABS_HD void eval_neighbours_r(const WalkState<W, T> &st, const Geometry &g, const Muls &mu, const uint32_t *mt, int tp,
                               int jprev, uint32_t floor, uint32_t (&top)[K]) {
  constexpr int T3 = T - 3 >= 2 ? T - 3 : 2;
  if (tp >= T) eval_neighbours_tp<W, T, T, K, RESCAN, PMAX, U>(st, g, mu, mt, jprev, floor, top);
  else if (tp == T - 1) eval_neighbours_tp<W, T, T - 1, K, RESCAN, PMAX, U>(st, g, mu, mt, jprev, floor, top);
  else if (tp == T - 2) eval_neighbours_tp<W, T, T - 2, K, RESCAN, PMAX, U>(st, g, mu, mt, jprev, floor, top);
  else eval_neighbours_tp<W, T, T3, K, RESCAN, PMAX, U>(st, g, mu, mt, jprev, floor, top);
}

template <int W, int T, int K, int PMAX, int U = 1>
LABS_HD void eval_neighbours(const WalkState<W, T> &st, const Geometry &g, const Muls &mu, const uint32_t *mt, int tp,
                             int jprev, uint32_t floor, uint32_t (&top)[K]) {
  if (floor == 0) eval_neighbours_r<W, T, K, false, PMAX, U>(st, g, mu, mt, tp, jprev, 0u, top);
  else eval_neighbours_r<W, T, K, true, PMAX, U>(st, g, mu, mt, tp, jprev, floor, top);
}

LABS_HD int key_flip(uint32_t k) { return (int)(k & 0xFFu); }
LABS_HD int key_delta(uint32_t k) { return (int)(k >> 8) - kDeltaBias; }

// The move's update of the digit planes (Algorithm 2, the move): C_{2i} -= 4
// u_i for the flip a with position bit ba, its y window F (class bits t+1, t+2,
// ...) and x window X (class bits t-1, t-2, ...; only the lags it holds are
// read), as a bit-sliced add of 2 d, d = -u / 2 in {-2..2}; E += delta.
template <int W, int T>
LABS_HD void move_planes(WalkState<W, T> &st, const Geometry &g, int a, int delta, uint32_t ba,
                         const uint32_t (&F)[W], const uint32_t (&X)[W]) {
  const int q = a & 1, t = a >> 1;
  const int Nq = g.D - q;  // class size N_q without indexing g.N
  const bool centre = (a == g.c);
  const uint32_t bm = 0u - ba;
  const int i0 = g.c - a;  // pair lag excluded from the y side
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t vx = low_mask_word(t, w);
    uint32_t vy = centre ? 0u : low_mask_word(Nq - 1 - t, w);
    if (!centre && ((i0 - 1) >> 5) == w) vy &= ~(1u << ((i0 - 1) & 31));
    const uint32_t Xw = X[w] ^ bm, Yw = F[w] ^ bm;
    // g_x = -x' in {-1,0,1}: bit0 = vx, sign bits = vx & ~X (X=1 -> +1, X=0 -> -1)
    const uint32_t x0 = vx, xs = vx & ~Xw;
    const uint32_t y0 = vy, ys = vy & ~Yw;
    // d = g_x + g_y in [-2, 2], three-bit two's complement
    const uint32_t d0 = x0 ^ y0;
    const uint32_t c1 = x0 & y0;
    const uint32_t d1 = xs ^ ys ^ c1;
    const uint32_t c2 = (xs & ys) | (c1 & (xs ^ ys));
    const uint32_t d2 = xs ^ ys ^ c2;
    // e += 2 d over T planes (addend planes: 0, d0, d1, d2, d2, ...)
    uint32_t carry = 0;
#pragma unroll
    for (int tt = 1; tt < T; ++tt) {
      const uint32_t add = tt == 1 ? d0 : (tt == 2 ? d1 : d2);
      const uint32_t e = st.ep[tt][w];
      st.ep[tt][w] = lop3<kLutXor3>(e, add, carry);
      carry = lop3<kLutMajority>(e, add, carry);
    }
  }
  st.E += delta;
}

// The move's bit flips: position a and its mirror (Eq. 2) in the parity
// classes, bit a of the key.
template <int W, int T>
LABS_HD void move_bits(WalkState<W, T> &st, const Geometry &g, int a) {
  constexpr int NS = W + 1;
  const int q = a & 1, t = a >> 1;
  const uint32_t mq = sel_mask(q != 0);
  uint32_t cq[NS];  // the flip's parity class, selected without dynamic indexing
#pragma unroll
  for (int w = 0; w < NS; ++w) cq[w] = (st.cls[1][w] & mq) | (st.cls[0][w] & ~mq);
  xor_bit(cq, t, 1u);
  if (a != g.c) xor_bit(cq, (g.L - 1 - a - q) >> 1, 1u);
#pragma unroll
  for (int w = 0; w < NS; ++w) {
    st.cls[0][w] = (st.cls[0][w] & mq) | (cq[w] & ~mq);
    st.cls[1][w] = (cq[w] & mq) | (st.cls[1][w] & ~mq);
  }
  xor_bit(st.key, a, 1u);
}

// Move to the neighbour of flip a (Algorithm 2, the move): cut the flip's
// windows from its parity class, update the planes and E, flip the bits.
template <int W, int T>
LABS_HD void apply_move(WalkState<W, T> &st, const Geometry &g, int a, int delta) {
  constexpr int NS = W + 1;
  const int q = a & 1, t = a >> 1;
  uint32_t cq[NS];  // the flip's parity class, selected without dynamic indexing
  const uint32_t mq = sel_mask(q != 0);
#pragma unroll
  for (int w = 0; w < NS; ++w) cq[w] = (st.cls[1][w] & mq) | (st.cls[0][w] & ~mq);
  const uint32_t ba = get_bit(cq, t);
  // Y window: class bits t+1 .. ; X window: class bits t-1, t-2, .. via a full bit reversal
  uint32_t F[W], R[NS], X[W];
  shr_dyn(F, cq, t + 1);
#pragma unroll
  for (int w = 0; w < NS; ++w) R[w] = brev32(cq[NS - 1 - w]);
  shr_dyn(X, R, 32 * NS - t);
  move_planes(st, g, a, delta, ba, F, X);
  // the bit flips on the class already selected (move_bits without its selection)
  xor_bit(cq, t, 1u);
  if (a != g.c) xor_bit(cq, (g.L - 1 - a - q) >> 1, 1u);
#pragma unroll
  for (int w = 0; w < NS; ++w) {
    st.cls[0][w] = (st.cls[0][w] & mq) | (cq[w] & ~mq);
    st.cls[1][w] = (cq[w] & mq) | (st.cls[1][w] & ~mq);
  }
  xor_bit(st.key, a, 1u);
}

// ------------------------------------------------------ visited hash table
// Open addressing with linear probing over `cap` (power of two) slots of
// KW64 64-bit words; a slot stores the D key bits plus an occupancy flag at
// bit D, and an all-zero slot is empty.  The hash is the MurmurHash3 32-bit
// finaliser (Appleby) applied to a multiplicative fold of the key words.
template <int NS>
LABS_HD uint32_t hash_key(const uint32_t (&k)[NS]) {
  uint32_t h = 0x2545F491u;
#pragma unroll
  for (int w = 0; w < NS; ++w) h = (h ^ k[w]) * 0x9E3779B1u + (uint32_t)w;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Look key up in the table; returns true if present, else false with *slot =
// the empty slot where it would be inserted.  *probes counts slots read;
// returns false with *slot = kNone if the table is full (cannot happen when
// cap exceeds the walk's pivot count, but is reported as an overflow).
template <int NS>
LABS_HD bool table_find(const uint64_t *table, uint32_t cap, int KW64, const uint32_t (&k)[NS], int D,
                        uint32_t *slot) {
  uint64_t want[(NS + 1) / 2 + 1];
#pragma unroll
  for (int i = 0; i < (NS + 1) / 2 + 1; ++i) {
    const uint32_t lo = 2 * i < NS ? k[2 * i] : 0u;
    const uint32_t hi = 2 * i + 1 < NS ? k[2 * i + 1] : 0u;
    want[i] = ((uint64_t)hi << 32) | lo;
  }
  // occupancy flag at bit D
#pragma unroll
  for (int i = 0; i < (NS + 1) / 2 + 1; ++i) want[i] |= ((D >> 6) == i) ? (1ull << (D & 63)) : 0ull;
  uint32_t idx = hash_key(k) & (cap - 1u);
  for (uint32_t n = 0; n < cap; ++n) {
    const uint64_t *s = table + (size_t)idx * KW64;
    bool empty = true, equal = true;
#pragma unroll
    for (int i = 0; i < (NS + 1) / 2 + 1; ++i) {
      if (i < KW64) {
        const uint64_t v = s[i];
        empty = empty && (v == 0);
        equal = equal && (v == want[i]);
      }
    }
    if (equal) return true;
    if (empty) {
      *slot = idx;
      return false;
    }
    idx = (idx + 1u) & (cap - 1u);
  }
  *slot = kNone;
  return false;
}

template <int NS>
LABS_HD void table_store(uint64_t *table, uint32_t slot, int KW64, const uint32_t (&k)[NS], int D) {
  uint64_t *s = table + (size_t)slot * KW64;
#pragma unroll
  for (int i = 0; i < (NS + 1) / 2 + 1; ++i) {
    if (i < KW64) {
      const uint32_t lo = 2 * i < NS ? k[2 * i] : 0u;
      const uint32_t hi = 2 * i + 1 < NS ? k[2 * i + 1] : 0u;
      s[i] = (((uint64_t)hi << 32) | lo) | (((D >> 6) == i) ? (1ull << (D & 63)) : 0ull);
    }
  }
}

LABS_HD int key_words64(int D) { return (D + 1 + 63) / 64; }

// Bit of position a (0-based; 1 <-> -1) of the length-L sequence whose key is
// k: a skew key holds the D free values and Eq. 2 gives the rest,
// s_{c+i} = (-1)^i s_{c-i} with c = D-1; a full-space key is the sequence.
LABS_HD uint32_t sequence_bit(const uint32_t *k, int L, int a, bool full) {
  const int c = (L - 1) / 2;
  if (full || a <= c) return (k[a >> 5] >> (a & 31)) & 1u;
  const int i = a - c, src = c - i;
  return ((k[src >> 5] >> (src & 31)) & 1u) ^ (uint32_t)(i & 1);
}

}  // namespace psaw
