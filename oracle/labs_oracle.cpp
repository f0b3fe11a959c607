// Reference oracle for the skew-symmetric LABS self-avoiding-walk solver of
// Bošković, Herzog and Brest, "Parallel Self-Avoiding Walks for a
// Low-Autocorrelation Binary Sequences Problem" (arXiv 2210.15962).
//
// TEST INFRASTRUCTURE ONLY.  This file is a deliberately plain, slow CPU
// restatement of the paper's definitions.  Only the test suite, the smoke
// check and the CPU-baseline leg of the benchmark may load it; the product
// library never does.  It shares no code with the CUDA path.
//
// Conventions (the paper's, with 0-based array indices):
//   * a sequence is s[0..L-1] with s[i] in {+1,-1}; s[i] is the paper's s_{i+1};
//   * Eq. 1:  C_k = sum_{i=1}^{L-k} s_i s_{i+k},  E = sum_{k=1}^{L-1} C_k^2,
//             F = L^2 / (2E);
//   * Eq. 2:  skew symmetry s_{D+i} = (-1)^i s_{D-i}, i = 1..D-1, D = (L+1)/2,
//             so the first D values are free and the rest follow from them;
//   * a flip j (0 <= j < D) negates free value s_{j+1} and therefore also its
//             mirror s_{L-j} (the same position when j = D-1, the centre);
//   * the full search space (all 2^L sequences, any L; the solver the paper
//             leaves to future work in Section 5): all L values are free, a
//             flip j (0 <= j < L) negates s_{j+1} alone, and the key of a
//             pivot is the whole sequence;
//   * bit convention for starts, keys and hex strings: bit 1 <-> -1, 0 <-> +1.
//
// Parity status: every function here is pinned by tests that do not call
// this code's own formulas again (Table 1 energies, closed forms, brute-force
// enumeration, Random123 known-answer vectors, invariants).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <set>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- Eq. 1
// C_k(S) = sum over i of s_i * s_{i+k}, for 0 <= k < L.
int64_t autocorrelation(const int8_t *s, int L, int k) {
  int64_t c = 0;
  for (int i = 0; i + k < L; ++i) c += (int64_t)s[i] * (int64_t)s[i + k];
  return c;
}

// E(S) = sum_{k=1}^{L-1} C_k^2 (Eq. 1).
int64_t energy_eq1(const int8_t *s, int L) {
  int64_t e = 0;
  for (int k = 1; k < L; ++k) {
    int64_t c = autocorrelation(s, L, k);
    e += c * c;
  }
  return e;
}

// ---------------------------------------------------------------- Eq. 2
// Fill s[D..L-1] from the free values s[0..D-1]:  s_{D+i} = (-1)^i s_{D-i}.
// With 0-based indices the centre is c = D-1 and s[c+i] = (-1)^i s[c-i].
void skew_expand(int8_t *s, int L) {
  const int D = (L + 1) / 2;
  const int c = D - 1;
  for (int i = 1; i <= D - 1; ++i) s[c + i] = (int8_t)((i & 1) ? -s[c - i] : s[c - i]);
}

// ------------------------------------------------------ Philox4x32-10 RNG
// The counter-based generator of Salmon, Moraes, Dror and Shaw, "Parallel
// random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of a 4x32-bit
// multiply/xor bijection keyed by a 2x32-bit key that is advanced by the Weyl
// constants between rounds.
struct P4 { uint32_t v[4]; };

P4 philox_round(P4 x, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * x.v[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * x.v[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  P4 y;
  y.v[0] = hi1 ^ x.v[1] ^ k0;
  y.v[1] = lo1;
  y.v[2] = hi0 ^ x.v[3] ^ k1;
  y.v[3] = lo0;
  return y;
}

P4 philox4x32_10(P4 ctr, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    ctr = philox_round(ctr, k0, k1);
  }
  return ctr;
}

// Random first pivot P_1 of Eq. 3 (the paper's rand{-1,+1} per free value).
// Stream layout: key = (seed low 32 bits, seed high 32 bits); block b of the
// stream is Philox(counter = (walk, round, b, 0)); free value j takes bit
// (j mod 32) of word ((j / 32) mod 4) of block (j / 128); bit 1 means -1.
void start_free_values(uint64_t seed, uint32_t walk, uint32_t round, int D, int8_t *free_out) {
  for (int j = 0; j < D; ++j) {
    P4 ctr = {{walk, round, (uint32_t)(j / 128), 0u}};
    P4 r = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t word = r.v[(j / 32) % 4];
    free_out[j] = ((word >> (j % 32)) & 1u) ? (int8_t)-1 : (int8_t)1;
  }
}

// ----------------------------------------------- one contiguous SAW (Eq. 3)
struct WalkResult {
  int64_t best_E = 0;
  std::vector<int8_t> best_seq;  // length L
  int32_t best_step = 0;         // pivot index (0 = P_1) where best_E was first reached
  int32_t moves = 0;             // moves made (pivots after P_1)
  int32_t stuck = 0;             // 1 if a step found every neighbour visited
  int64_t evals = 0;             // neighbour evaluations performed
};

using Key = std::vector<int8_t>;  // the D free values identify a skew pivot

Key key_of(const std::vector<int8_t> &s, int D) { return Key(s.begin(), s.begin() + D); }

// The search space of a walk: the skew-symmetric sequences (D free values,
// flip j negates positions j and L-1-j) or all sequences (L free values, flip
// j negates position j).
struct Space {
  bool full;
  int L;
  int free_values() const { return full ? L : (L + 1) / 2; }
  int mirror(int j) const { return full ? j : L - 1 - j; }
};

// Change of C_k (k = 1..L-1) when the positions in {p, q} are negated.
// A product s_i s_{i+k} changes sign iff exactly one of its two positions is
// negated, so dC_k = sum of -2 s_i s_{i+k} over those pairs.  This is the
// plain O(1)-per-lag incremental update of the sidelobe array that the
// paper's fast neighbourhood evaluation relies on.
void sidelobe_change(const std::vector<int8_t> &s, int L, int p, int q, std::vector<int64_t> &dC) {
  for (int k = 1; k < L; ++k) {
    int64_t d = 0;
    const int cand[4] = {p, q, p - k, q - k};
    int seen[4];
    int ns = 0;
    for (int t = 0; t < 4; ++t) {
      const int i = cand[t];
      if (i < 0 || i + k >= L) continue;
      bool dup = false;
      for (int u = 0; u < ns; ++u) dup |= (seen[u] == i);
      if (dup) continue;
      seen[ns++] = i;
      const bool a = (i == p || i == q);
      const bool b = (i + k == p || i + k == q);
      if (a != b) d += -2 * (int64_t)s[i] * (int64_t)s[i + k];
    }
    dC[k] = d;
  }
}

// One contiguous self-avoiding walk of Eq. 3 / Algorithm 2 for walk index
// `walk` of round `round` of the problem seeded by `seed`.
//   * P_1 is drawn by start_free_values and expanded by Eq. 2;
//   * every step evaluates all D neighbours (flips) with the incremental
//     sidelobe update, skips neighbours equal to an earlier pivot of this walk
//     (exact std::set of full keys), and moves to the lowest-energy one, the
//     lowest flip index winning ties;
//   * a walk whose neighbours are all visited stops ("stuck");
//   * the walk's best (E, sequence) is replaced only on strict improvement.
// When `check` is set every neighbour energy and every new pivot's energy and
// sidelobe array are also recomputed from Eq. 1 and compared (aborting on a
// mismatch).  `flips_out` (walk_len entries) and `energy_out` (walk_len + 1
// entries) optionally record the trajectory.
WalkResult run_walk(const Space &sp, uint64_t seed, uint32_t walk, uint32_t round, int walk_len, bool check,
                    int32_t *flips_out, int64_t *energy_out, int *check_failed) {
  const int L = sp.L;
  const int D = sp.free_values();  // flips per step and length of a key
  std::vector<int8_t> s(L);
  start_free_values(seed, walk, round, D, s.data());
  if (!sp.full) skew_expand(s.data(), L);

  std::vector<int64_t> C(L);
  for (int k = 0; k < L; ++k) C[k] = autocorrelation(s.data(), L, k);
  int64_t E = 0;
  for (int k = 1; k < L; ++k) E += C[k] * C[k];

  std::set<Key> visited;
  visited.insert(key_of(s, D));

  WalkResult res;
  res.best_E = E;
  res.best_seq = s;
  res.best_step = 0;
  if (energy_out) energy_out[0] = E;

  std::vector<int64_t> dC(L), best_dC(L);
  std::vector<int8_t> nb(L);
  for (int step = 1; step <= walk_len; ++step) {
    int best_j = -1;
    int64_t best_delta = 0;
    for (int j = 0; j < D; ++j) {
      const int p = j, q = sp.mirror(j);
      sidelobe_change(s, L, p, q, dC);
      int64_t delta = 0;
      for (int k = 1; k < L; ++k) delta += (C[k] + dC[k]) * (C[k] + dC[k]) - C[k] * C[k];
      if (check) {
        nb = s;
        nb[p] = (int8_t)-nb[p];
        if (q != p) nb[q] = (int8_t)-nb[q];
        if (energy_eq1(nb.data(), L) - E != delta) *check_failed = 1;
      }
      Key nk = key_of(s, D);
      nk[j] = (int8_t)-nk[j];
      if (visited.count(nk)) continue;
      if (best_j < 0 || delta < best_delta) {
        best_j = j;
        best_delta = delta;
        best_dC = dC;
      }
    }
    res.evals += D;
    if (best_j < 0) {
      res.stuck = 1;
      break;
    }
    const int p = best_j, q = sp.mirror(best_j);
    s[p] = (int8_t)-s[p];
    if (q != p) s[q] = (int8_t)-s[q];
    for (int k = 1; k < L; ++k) C[k] += best_dC[k];
    E += best_delta;
    visited.insert(key_of(s, D));
    res.moves = step;
    if (flips_out) flips_out[step - 1] = best_j;
    if (energy_out) energy_out[step] = E;
    if (check) {
      if (energy_eq1(s.data(), L) != E) *check_failed = 1;
      for (int k = 1; k < L; ++k)
        if (autocorrelation(s.data(), L, k) != C[k]) *check_failed = 1;
    }
    if (E < res.best_E) {
      res.best_E = E;
      res.best_seq = s;
      res.best_step = step;
    }
  }
  return res;
}

}  // namespace

extern "C" {

// Eq. 1 energy of an arbitrary +-1 sequence.  Returns -1 on bad arguments.
int64_t oracle_energy(const int8_t *s, int32_t L) {
  if (!s || L < 1) return -1;
  for (int i = 0; i < L; ++i)
    if (s[i] != 1 && s[i] != -1) return -1;
  return energy_eq1(s, L);
}

// All C_k, k = 0..L-1, of Eq. 1.
int32_t oracle_autocorrelations(const int8_t *s, int32_t L, int64_t *C_out) {
  if (!s || !C_out || L < 1) return -1;
  for (int k = 0; k < L; ++k) C_out[k] = autocorrelation(s, L, k);
  return 0;
}

// Eq. 2: write the length-L skew-symmetric sequence whose first D values are
// free_vals.  Returns -1 unless L is odd and >= 3.
int32_t oracle_skew_expand(const int8_t *free_vals, int32_t L, int8_t *seq_out) {
  if (!free_vals || !seq_out || L < 3 || (L % 2) == 0) return -1;
  const int D = (L + 1) / 2;
  std::memcpy(seq_out, free_vals, (size_t)D);
  skew_expand(seq_out, L);
  return 0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  P4 c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
  P4 r = philox4x32_10(c, key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

void oracle_start_free_values(uint64_t seed, uint32_t walk, uint32_t round, int32_t D, int8_t *free_out) {
  start_free_values(seed, walk, round, D, free_out);
}

// One walk with its trajectory.  flips_out: walk_len int32 (the flip chosen at
// each step), energy_out: walk_len + 1 int64 (E of P_1 .. P_{walk_len+1}),
// best_seq_out: L int8.  Returns 0, or 1 if check mode found a mismatch, or
// -1 on bad arguments.  Any of the output pointers may be null.
static int32_t walk_trace_impl(const Space &sp, uint64_t seed, uint32_t walk, uint32_t round, int32_t walk_len,
                               int32_t check, int32_t *flips_out, int64_t *energy_out, int8_t *best_seq_out,
                               int64_t *best_E_out, int32_t *moves_out, int32_t *stuck_out, int32_t *best_step_out) {
  int failed = 0;
  WalkResult r = run_walk(sp, seed, walk, round, walk_len, check != 0, flips_out, energy_out, &failed);
  if (best_seq_out) std::memcpy(best_seq_out, r.best_seq.data(), (size_t)sp.L);
  if (best_E_out) *best_E_out = r.best_E;
  if (moves_out) *moves_out = r.moves;
  if (stuck_out) *stuck_out = r.stuck;
  if (best_step_out) *best_step_out = r.best_step;
  return failed ? 1 : 0;
}

int32_t oracle_walk_trace(int32_t L, uint64_t seed, uint32_t walk, uint32_t round, int32_t walk_len,
                          int32_t check, int32_t *flips_out, int64_t *energy_out, int8_t *best_seq_out,
                          int64_t *best_E_out, int32_t *moves_out, int32_t *stuck_out, int32_t *best_step_out) {
  if (L < 5 || (L % 2) == 0 || walk_len < 0) return -1;
  return walk_trace_impl(Space{false, L}, seed, walk, round, walk_len, check, flips_out, energy_out, best_seq_out,
                         best_E_out, moves_out, stuck_out, best_step_out);
}

// The same walk over the full search space (any L >= 2).
int32_t oracle_full_walk_trace(int32_t L, uint64_t seed, uint32_t walk, uint32_t round, int32_t walk_len,
                               int32_t check, int32_t *flips_out, int64_t *energy_out, int8_t *best_seq_out,
                               int64_t *best_E_out, int32_t *moves_out, int32_t *stuck_out, int32_t *best_step_out) {
  if (L < 2 || walk_len < 0) return -1;
  return walk_trace_impl(Space{true, L}, seed, walk, round, walk_len, check, flips_out, energy_out, best_seq_out,
                         best_E_out, moves_out, stuck_out, best_step_out);
}

// A batch of walks [walk_begin, walk_begin + n_walks) of one round, run on
// `threads` host threads.  Per walk: best E, best sequence (L int8), moves,
// stuck flag, neighbour evaluations.
static int32_t walk_batch_impl(const Space &sp, uint64_t seed, uint32_t round, uint32_t walk_begin,
                               int32_t n_walks, int32_t walk_len, int32_t threads, int64_t *best_E,
                               int8_t *best_seq, int32_t *moves, int32_t *stuck, int64_t *evals) {
  const int L = sp.L;
  if (threads < 1) threads = 1;
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) {
    pool.emplace_back([=]() {
      for (int w = t; w < n_walks; w += threads) {
        int failed = 0;
        WalkResult r = run_walk(sp, seed, walk_begin + (uint32_t)w, round, walk_len, false, nullptr, nullptr, &failed);
        if (best_E) best_E[w] = r.best_E;
        if (best_seq) std::memcpy(best_seq + (size_t)w * L, r.best_seq.data(), (size_t)L);
        if (moves) moves[w] = r.moves;
        if (stuck) stuck[w] = r.stuck;
        if (evals) evals[w] = r.evals;
      }
    });
  }
  for (auto &th : pool) th.join();
  return 0;
}

int32_t oracle_walk_batch(int32_t L, uint64_t seed, uint32_t round, uint32_t walk_begin, int32_t n_walks,
                          int32_t walk_len, int32_t threads, int64_t *best_E, int8_t *best_seq,
                          int32_t *moves, int32_t *stuck, int64_t *evals) {
  if (L < 5 || (L % 2) == 0 || walk_len < 0 || n_walks < 0) return -1;
  return walk_batch_impl(Space{false, L}, seed, round, walk_begin, n_walks, walk_len, threads, best_E, best_seq,
                         moves, stuck, evals);
}

int32_t oracle_full_walk_batch(int32_t L, uint64_t seed, uint32_t round, uint32_t walk_begin, int32_t n_walks,
                               int32_t walk_len, int32_t threads, int64_t *best_E, int8_t *best_seq,
                               int32_t *moves, int32_t *stuck, int64_t *evals) {
  if (L < 2 || walk_len < 0 || n_walks < 0) return -1;
  return walk_batch_impl(Space{true, L}, seed, round, walk_begin, n_walks, walk_len, threads, best_E, best_seq,
                         moves, stuck, evals);
}

// The whole solve of Algorithm 1 for each of n_seeds independent problems:
// rounds r = 0, 1, ... each run `walks` contiguous SAWs; after each round the
// problem's best is the minimum over walks by (E, round, walk); rounds go on
// while the neighbour evaluations done are below step_budget and (when
// target_E >= 0) the best E is above target_E.  Outputs per seed: best_E,
// best_seq (L int8), evals done, rounds run.
static int32_t solve_impl(const Space &sp, const uint64_t *seeds, int32_t n_seeds, int32_t walks, int32_t walk_len,
                          uint64_t step_budget, int64_t target_E, int32_t threads, int64_t *best_E,
                          int8_t *best_seq, uint64_t *evals_out, int32_t *rounds_out) {
  const int L = sp.L;
  std::vector<int64_t> bE(walks), ev(walks);
  std::vector<int8_t> bS((size_t)walks * L);
  for (int si = 0; si < n_seeds; ++si) {
    uint64_t done = 0;
    int64_t cur = -1;
    std::vector<int8_t> cur_seq(L);
    uint32_t round = 0;
    for (;;) {
      walk_batch_impl(sp, seeds[si], round, 0, walks, walk_len, threads, bE.data(), bS.data(), nullptr, nullptr,
                      ev.data());
      for (int w = 0; w < walks; ++w) {
        done += (uint64_t)ev[w];
        if (cur < 0 || bE[w] < cur) {
          cur = bE[w];
          std::memcpy(cur_seq.data(), bS.data() + (size_t)w * L, (size_t)L);
        }
      }
      ++round;
      if (done >= step_budget) break;
      if (target_E >= 0 && cur <= target_E) break;
    }
    if (best_E) best_E[si] = cur;
    if (best_seq) std::memcpy(best_seq + (size_t)si * L, cur_seq.data(), (size_t)L);
    if (evals_out) evals_out[si] = done;
    if (rounds_out) rounds_out[si] = (int32_t)round;
  }
  return 0;
}

int32_t oracle_solve(int32_t L, const uint64_t *seeds, int32_t n_seeds, int32_t walks, int32_t walk_len,
                     uint64_t step_budget, int64_t target_E, int32_t threads, int64_t *best_E,
                     int8_t *best_seq, uint64_t *evals_out, int32_t *rounds_out) {
  if (L < 5 || (L % 2) == 0 || walks < 1 || walk_len < 0 || step_budget == 0 || !seeds) return -1;
  return solve_impl(Space{false, L}, seeds, n_seeds, walks, walk_len, step_budget, target_E, threads, best_E,
                    best_seq, evals_out, rounds_out);
}

int32_t oracle_full_solve(int32_t L, const uint64_t *seeds, int32_t n_seeds, int32_t walks, int32_t walk_len,
                          uint64_t step_budget, int64_t target_E, int32_t threads, int64_t *best_E,
                          int8_t *best_seq, uint64_t *evals_out, int32_t *rounds_out) {
  if (L < 2 || walks < 1 || walk_len < 0 || step_budget == 0 || !seeds) return -1;
  return solve_impl(Space{true, L}, seeds, n_seeds, walks, walk_len, step_budget, target_E, threads, best_E,
                    best_seq, evals_out, rounds_out);
}

}  // extern "C"
