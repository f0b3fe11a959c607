// Runs the CUDA path's walk cores on the host: walk_core.cuh, full_core.cuh
// and walk_incr.cuh hold the arithmetic of the walk kernels as host+device
// functions, and this program compiles them with the host compiler.  It reads
// cases from stdin, one per line:
//   skew L seed round walk walk_len force_tp pmax
//   full L seed round walk walk_len force_tp
//   incr L seed round walk walk_len            (the incremental neighbourhood)
// and prints, per case, one line
//   moves stuck best_E recheck_ok | flip_1 .. flip_moves | E_0 E_1 .. E_moves
// A CPU test compares these with the oracle walk by walk.  The step loop here
// (best of the 4 smallest keys by probing the visited table in key order,
// a rescan above the 4th key when all 4 are visited) restates the kernels'
// step; its scan, move, plane-count, start and table functions are the
// kernels' own.  force_tp = 1 scans with all T digit planes instead of the
// fewest that hold every C; pmax is the widest lag-word class that scans in
// pattern runs (3 in the per-round and the persistent batch kernels; 2 and 4
// exercise the same templates one class narrower and wider).
#include <cstdint>
#include <cstdio>
#include <iostream>
#include <sstream>
#include <string>
#include <type_traits>
#include <vector>

#include "walk_core.cuh"
#include "full_core.cuh"
#include "walk_incr.cuh"

using namespace psaw;

namespace {

struct Walk {
  std::vector<int> flips;
  std::vector<long long> energies;
  int best_E = 0;
  int stuck = 0;
  bool recheck_ok = true;
};

constexpr int kTop = 4;

// visited-table capacity: a power of two above 1.5x the walk's pivots
uint32_t table_cap(int walk_len) {
  uint32_t cap = 64;
  while (cap < (uint32_t)((walk_len + 1) * 3 / 2 + 1)) cap <<= 1;
  return cap;
}

// The move of one step: the smallest unvisited key among the candidates of
// eval(floor), rescanning above the 4th while all 4 are visited.
template <int NS, class Eval>
bool choose(Eval &&eval, const uint32_t (&key)[NS], int D, const std::vector<uint64_t> &table, uint32_t cap, int kw,
            int *flip, int *delta, uint32_t *slot) {
  uint32_t floor = 0;
  for (;;) {
    uint32_t top[kTop];
    eval(floor, top);
    for (int r = 0; r < kTop; ++r) {
      if (top[r] == kNone) return false;
      uint32_t nk[NS];
      for (int w = 0; w < NS; ++w) nk[w] = key[w];
      xor_bit(nk, key_flip(top[r]), 1u);
      uint32_t s;
      if (!table_find(table.data(), cap, kw, nk, D, &s)) {
        *flip = key_flip(top[r]);
        *delta = key_delta(top[r]);
        *slot = s;
        return true;
      }
    }
    floor = top[kTop - 1] + 1;
  }
}

// the digit planes the walk kernels use for lag-word class W
template <int W>
constexpr int skew_planes() {
  return W == 1 ? 6 : (W == 2 ? 7 : (W <= 4 ? 8 : 9));
}

template <int W, int PMAX>
Walk run_skew(int L, uint64_t seed, uint32_t walk, uint32_t round, int walk_len, bool force_tp) {
  constexpr int T = skew_planes<W>();
  constexpr int NS = W + 1;
  const Geometry g = make_geometry(L, T);
  std::vector<uint32_t> mt(MaskTable<W>::kWords);
  fill_mask_rows<W>(g, mt.data(), 0, 1);
  WalkState<W, T> st;
  init_walk(st, g, seed, walk, round);
  Walk out;
  out.recheck_ok = recheck_walk(st, g);
  const uint32_t cap = table_cap(walk_len);
  const int kw = key_words64(g.D);
  std::vector<uint64_t> table((size_t)cap * kw, 0);
  uint32_t slot;
  table_find(table.data(), cap, kw, st.key, g.D, &slot);
  table_store(table.data(), slot, kw, st.key, g.D);
  out.best_E = st.E;
  out.energies.push_back(st.E);
  const Muls mu{1u, 2u, 4u, 0x80000000u, 0x40000000u};
  int jprev = -1;
  for (int step = 1; step <= walk_len; ++step) {
    const int tp = force_tp ? T : planes_needed(st, g);
    auto eval = [&](uint32_t floor, uint32_t (&top)[kTop]) {
      eval_neighbours<W, T, kTop, PMAX>(st, g, mu, mt.data(), tp, jprev, floor, top);
    };
    int flip, delta;
    if (!choose<NS>(eval, st.key, g.D, table, cap, kw, &flip, &delta, &slot)) {
      out.stuck = 1;
      break;
    }
    apply_move(st, g, flip, delta);
    table_store(table.data(), slot, kw, st.key, g.D);
    jprev = flip;
    out.flips.push_back(flip);
    out.energies.push_back(st.E);
    out.recheck_ok = out.recheck_ok && recheck_walk(st, g);
    if (st.E < out.best_E) out.best_E = st.E;
  }
  return out;
}

template <int W>
Walk run_full(int L, uint64_t seed, uint32_t walk, uint32_t round, int walk_len, bool force_tp) {
  constexpr int T = FullPlanesFor<W>::value;
  constexpr int NS = W + 1;
  std::vector<uint32_t> mt(FullMaskTable<W>::kWords);
  fill_full_mask_rows<W>(L, mt.data(), 0, 1);
  FullState<W, T> st;
  init_full(st, L, seed, walk, round);
  Walk out;
  out.recheck_ok = recheck_full(st, L);
  const uint32_t cap = table_cap(walk_len);
  const int kw = key_words64(L);
  std::vector<uint64_t> table((size_t)cap * kw, 0);
  uint32_t slot;
  table_find(table.data(), cap, kw, st.bits, L, &slot);
  table_store(table.data(), slot, kw, st.bits, L);
  out.best_E = st.E;
  out.energies.push_back(st.E);
  const Muls mu{1u, 2u, 4u, 0x80000000u, 0x40000000u};
  int jprev = -1;
  for (int step = 1; step <= walk_len; ++step) {
    const int tp = force_tp ? T : full_planes_needed(st, L);
    auto eval = [&](uint32_t floor, uint32_t (&top)[kTop]) {
      full_eval<W, T, kTop>(st, L, mu, mt.data(), tp, jprev, floor, top);
    };
    int flip, delta;
    if (!choose<NS>(eval, st.bits, L, table, cap, kw, &flip, &delta, &slot)) {
      out.stuck = 1;
      break;
    }
    apply_full(st, L, flip, delta);
    table_store(table.data(), slot, kw, st.bits, L);
    jprev = flip;
    out.flips.push_back(flip);
    out.energies.push_back(st.E);
    out.recheck_ok = out.recheck_ok && recheck_full(st, L);
    if (st.E < out.best_E) out.best_E = st.E;
  }
  return out;
}

// the incremental variant's storage per class, as its kernel stores it:
// C_{2i} as int8 up to two lag words, Delta / 8 as int16 up to three
template <int W>
struct IncrStorage {
  using CT = typename std::conditional<W <= 2, int8_t, int16_t>::type;
  using DT = typename std::conditional<W <= 3, int16_t, int32_t>::type;
};

template <int W>
Walk run_incr(int L, uint64_t seed, uint32_t walk, uint32_t round, int walk_len) {
  using CT = typename IncrStorage<W>::CT;
  using DT = typename IncrStorage<W>::DT;
  constexpr int NS = W + 1;
  const Geometry g = make_geometry(L, skew_planes<W>());
  std::vector<CT> Cs(g.m + 1);
  std::vector<DT> Ds(g.D + 1);
  const IncrView<CT, DT> v{Cs.data(), Ds.data(), 1};
  IncrState<W> st;
  init_incr(st, g, v, seed, walk, round);
  Walk out;
  out.recheck_ok = recheck_incr(st, g, v);
  const uint32_t cap = table_cap(walk_len);
  const int kw = key_words64(g.D);
  std::vector<uint64_t> table((size_t)cap * kw, 0);
  uint32_t slot;
  table_find(table.data(), cap, kw, st.key, g.D, &slot);
  table_store(table.data(), slot, kw, st.key, g.D);
  out.best_E = st.E;
  out.energies.push_back(st.E);
  const Muls mu{1u, 2u, 4u, 0x80000000u, 0x40000000u};
  int jprev = -1;
  // the stored deltas are scanned once at the start; each move updates them
  // and hands over the next step's 4 smallest keys; rescans read them again
  uint32_t next[kTop];
  scan_stored<W, CT, DT, kTop>(g, v, -1, 0u, next);
  for (int step = 1; step <= walk_len; ++step) {
    auto eval = [&](uint32_t floor, uint32_t (&top)[kTop]) {
      if (floor == 0) {
        for (int r = 0; r < kTop; ++r) top[r] = next[r];
      } else {
        scan_stored<W, CT, DT, kTop>(g, v, jprev, floor, top);
      }
    };
    int flip, delta;
    const bool found = choose<NS>(eval, st.key, g.D, table, cap, kw, &flip, &delta, &slot);
    if (!found) {
      out.stuck = 1;
      break;
    }
    MoveData<W> md;
    apply_move_incr(st, g, v, flip, md);
    table_store(table.data(), slot, kw, st.key, g.D);
    jprev = flip;
    out.flips.push_back(flip);
    out.energies.push_back(st.E);
    if (st.E < out.best_E) out.best_E = st.E;
    update_neighbours_fast<W, CT, DT, kTop>(st, g, v, md, mu, next);
    out.recheck_ok = out.recheck_ok && recheck_incr(st, g, v);
  }
  return out;
}

Walk incr_by_class(int L, uint64_t seed, uint32_t round, uint32_t walk, int walk_len) {
  switch (((L - 1) / 2 + 31) / 32) {
    case 1: return run_incr<1>(L, seed, walk, round, walk_len);
    case 2: return run_incr<2>(L, seed, walk, round, walk_len);
    case 3: return run_incr<3>(L, seed, walk, round, walk_len);
    case 4: return run_incr<4>(L, seed, walk, round, walk_len);
    case 5: return run_incr<5>(L, seed, walk, round, walk_len);
    case 6: return run_incr<6>(L, seed, walk, round, walk_len);
    case 7: return run_incr<7>(L, seed, walk, round, walk_len);
    default: return run_incr<8>(L, seed, walk, round, walk_len);
  }
}

template <int PMAX>
Walk skew_by_class(int L, uint64_t seed, uint32_t round, uint32_t walk, int walk_len, bool force_tp) {
  switch (((L - 1) / 2 + 31) / 32) {
    case 1: return run_skew<1, PMAX>(L, seed, walk, round, walk_len, force_tp);
    case 2: return run_skew<2, PMAX>(L, seed, walk, round, walk_len, force_tp);
    case 3: return run_skew<3, PMAX>(L, seed, walk, round, walk_len, force_tp);
    case 4: return run_skew<4, PMAX>(L, seed, walk, round, walk_len, force_tp);
    case 5: return run_skew<5, PMAX>(L, seed, walk, round, walk_len, force_tp);
    case 6: return run_skew<6, PMAX>(L, seed, walk, round, walk_len, force_tp);
    case 7: return run_skew<7, PMAX>(L, seed, walk, round, walk_len, force_tp);
    default: return run_skew<8, PMAX>(L, seed, walk, round, walk_len, force_tp);
  }
}

Walk full_by_class(int L, uint64_t seed, uint32_t round, uint32_t walk, int walk_len, bool force_tp) {
  switch ((L - 1 + 31) / 32) {
    case 0:
    case 1: return run_full<1>(L, seed, walk, round, walk_len, force_tp);
    case 2: return run_full<2>(L, seed, walk, round, walk_len, force_tp);
    case 3: return run_full<3>(L, seed, walk, round, walk_len, force_tp);
    case 4: return run_full<4>(L, seed, walk, round, walk_len, force_tp);
    case 5: return run_full<5>(L, seed, walk, round, walk_len, force_tp);
    case 6: return run_full<6>(L, seed, walk, round, walk_len, force_tp);
    case 7: return run_full<7>(L, seed, walk, round, walk_len, force_tp);
    default: return run_full<8>(L, seed, walk, round, walk_len, force_tp);
  }
}

}  // namespace

int main() {
  std::string line;
  while (std::getline(std::cin, line)) {
    std::istringstream in(line);
    std::string space;
    int L = 0, walk_len = 0, force_tp = 0, pmax = 3;
    unsigned long long seed = 0;
    unsigned round = 0, walk = 0;
    if (!(in >> space >> L >> seed >> round >> walk >> walk_len)) continue;
    if (space != "incr" && !(in >> force_tp)) return 2;
    Walk r;
    if (space == "skew") {
      in >> pmax;
      if (L < kLMin || L > kLMax || (L % 2) == 0) return 2;
      r = pmax == 2   ? skew_by_class<2>(L, seed, round, walk, walk_len, force_tp != 0)
          : pmax == 3 ? skew_by_class<3>(L, seed, round, walk, walk_len, force_tp != 0)
                      : skew_by_class<4>(L, seed, round, walk, walk_len, force_tp != 0);
    } else if (space == "incr") {
      if (L < kLMin || L > kLMax || (L % 2) == 0) return 2;
      r = incr_by_class(L, seed, round, walk, walk_len);
    } else if (space == "full") {
      if (L < kFullLMin || L > kFullLMax) return 2;
      r = full_by_class(L, seed, round, walk, walk_len, force_tp != 0);
    } else {
      return 2;
    }
    std::printf("%zu %d %d %d |", r.flips.size(), r.stuck, r.best_E, r.recheck_ok ? 1 : 0);
    for (int f : r.flips) std::printf(" %d", f);
    std::printf(" |");
    for (long long e : r.energies) std::printf(" %lld", e);
    std::printf("\n");
  }
  return 0;
}
