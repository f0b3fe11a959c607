// Host side of the C ABI declared in include/labs.h: argument checks,
// workspace layout, the round loop of Algorithm 1 and result copies.  All
// arithmetic of the method runs in the kernels of walk_class.cu and walk_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/labs.h"
#include "walk_kernels.cuh"

namespace psaw {
namespace {

constexpr size_t kAlign = 256;
constexpr uint64_t kRoundBatch = 16;  // rounds enqueued between host checks of the stop flags

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool valid_L(int32_t L) { return L >= LABS_L_MIN && L <= LABS_L_MAX && (L & 1); }
bool valid_full_L(int32_t L) { return L >= LABS_FULL_L_MIN && L <= LABS_FULL_L_MAX; }
bool valid_space_L(int32_t space, int32_t L) { return space == kSpaceFull ? valid_full_L(L) : valid_L(L); }

// flips per step = bits of a key: D free values of a skew sequence, L of any sequence
int key_bits(int32_t space, int32_t L) { return space == kSpaceFull ? L : (L + 1) / 2; }
int space_lag_words(int32_t space, int32_t L) { return space == kSpaceFull ? full_lag_words(L) : lag_words(L); }

// visited-table slots: a power of two >= 3 x the pivots of a walk
uint32_t table_cap(int32_t walk_len) { return visited_table_cap(walk_len); }

// A bump allocator over one device block.
struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(void *b) : base((char *)b) {}
  template <typename T>
  T *take(size_t n) {
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off = align_up(off + n * sizeof(T));
    return p;
  }
};

struct Buffers {
  int32_t *w_bestE, *w_moves, *w_stuck, *w_best_step;
  uint32_t *w_key;
  unsigned long long *p_evals, *p_round_best;
  int64_t *p_bestE;
  uint32_t *p_key;
  int32_t *p_rounds, *p_best_round, *p_best_walk, *done;
  uint64_t *seeds, *budget;
  int64_t *target;
  int8_t *best_seq;
  int32_t *err;
  unsigned long long *plane_steps;
  uint64_t *tables;
};

// Lay out everything except the tables, then g_chunk tables.
size_t carve(Buffers &b, void *base, int L, int n_seeds, size_t n_walks, size_t g_chunk, size_t table_bytes) {
  Carver c(base);
  b.w_bestE = c.take<int32_t>(n_walks);
  b.w_moves = c.take<int32_t>(n_walks);
  b.w_stuck = c.take<int32_t>(n_walks);
  b.w_best_step = c.take<int32_t>(n_walks);
  b.w_key = c.take<uint32_t>(n_walks * kKeyWords);
  b.p_evals = c.take<unsigned long long>(n_seeds);
  b.p_round_best = c.take<unsigned long long>(n_seeds);
  b.p_bestE = c.take<int64_t>(n_seeds);
  b.p_key = c.take<uint32_t>((size_t)n_seeds * kKeyWords);
  b.p_rounds = c.take<int32_t>(n_seeds);
  b.p_best_round = c.take<int32_t>(n_seeds);
  b.p_best_walk = c.take<int32_t>(n_seeds);
  b.done = c.take<int32_t>(n_seeds);
  b.seeds = c.take<uint64_t>(n_seeds);
  b.budget = c.take<uint64_t>(n_seeds);
  b.target = c.take<int64_t>(n_seeds);
  b.best_seq = c.take<int8_t>((size_t)n_seeds * L);
  b.err = c.take<int32_t>(1);
  b.plane_steps = c.take<unsigned long long>(1);
  b.tables = c.take<uint64_t>(g_chunk * (table_bytes / 8));
  return c.off;
}

labs_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LABS_OK;
  if (e == cudaErrorMemoryAllocation) return LABS_ENOMEM;
  return LABS_ECUDA;
}

#define LABS_CU(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      st = cuda_status(e_);                             \
      goto done;                                        \
    }                                                   \
  } while (0)

// Event pairs around walk launches, summed at the end.
struct Timer {
  std::vector<cudaEvent_t> ev;
  cudaEvent_t rec(cudaStream_t s) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, s);
    ev.push_back(e);
    return e;
  }
  ~Timer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

double elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (a && b && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) return ms;
  return 0.0;
}

// Keep memory freed with cudaFreeAsync in this process's default pool of the
// current device instead of returning it to the driver at every
// synchronisation (a process-local allocator setting).
void retain_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  uint64_t keep = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
}

struct RunConfig {
  int32_t L, n_seeds, walks, walk_len, recheck_every;
  uint64_t budget;
  int64_t target;
  int32_t max_rounds;
  int32_t kernel;
  int32_t space;  // kSpaceSkew or kSpaceFull
};

// The neighbourhood evaluation of labs_opts.kernel (0 is resolved by
// Run::pick_variant before any round runs; the full scan stands in for it).
int32_t resolve_variant(int32_t kernel) {
  if (kernel == kVariantFullScan || kernel == kVariantIncremental || kernel == kVariantWarp ||
      kernel == kVariantCta)
    return kernel;
  return kVariantFullScan;
}

// The library's choice for labs_opts.kernel == 0 (skew space): one lane per
// walk, one warp per walk or (for launches of few walks) one CTA per walk,
// whichever ran a sample round of the same launch size faster, timed once per process for each lag-word class and launch size
// (log2 of the walks in one launch) by the first call whose walks have at least
// kSampleSteps steps (a call of shorter walks times a sample of its own
// length and keeps the choice to itself).  The incremental variant is never chosen:
// it measured slower than the full scan at every class (it pays a fixed
// per-flip cost at small W and its shared-memory state caps occupancy at
// large W).  Every variant gives the same results.
std::mutex g_variant_mu;
std::map<std::pair<int, int>, int32_t> g_variant;

int ilog2(uint64_t x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

constexpr int32_t kSampleSteps = 256;  // steps per walk of a variant-choice sample round
constexpr int kCtaMaxWalksPerSm = 16;  // largest launch (walks per SM) for which one CTA per walk is timed

}  // namespace
}  // namespace psaw

using namespace psaw;

extern "C" void labs_opts_init(labs_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->target_E = -1;
}

extern "C" const char *labs_status_str(labs_status s) {
  switch (s) {
    case LABS_OK: return "ok";
    case LABS_PENDING: return "pending";
    case LABS_EINVAL: return "invalid argument";
    case LABS_ENOMEM: return "out of device memory";
    case LABS_ECUDA: return "CUDA error";
    case LABS_ETIMEOUT: return "timeout";
    case LABS_EOVERFLOW: return "visited table overflow";
    case LABS_ENOTFOUND: return "unknown ticket";
    case LABS_ECHECK: return "recheck mismatch";
    case LABS_ESHUTDOWN: return "server shutting down";
    default: return "unknown status";
  }
}

extern "C" int64_t labs_energy(const int8_t *seq, int32_t L) {
  if (!seq || L < 1 || L > 65536) return LABS_EINVAL;
  int8_t *d_seq = nullptr;
  int64_t *d_E = nullptr;
  int32_t *d_err = nullptr;
  int64_t E = 0;
  int32_t err = 0;
  labs_status st = LABS_OK;
  LABS_CU(cudaMalloc(&d_seq, (size_t)L));
  LABS_CU(cudaMalloc(&d_E, sizeof(int64_t)));
  LABS_CU(cudaMalloc(&d_err, sizeof(int32_t)));
  LABS_CU(cudaMemcpy(d_seq, seq, (size_t)L, cudaMemcpyHostToDevice));
  LABS_CU(cudaMemset(d_err, 0, sizeof(int32_t)));
  LABS_CU(launch_energy(d_seq, 1, L, d_E, d_err, 0));
  LABS_CU(cudaMemcpy(&E, d_E, sizeof(int64_t), cudaMemcpyDeviceToHost));
  LABS_CU(cudaMemcpy(&err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (err) st = LABS_EINVAL;
done:
  cudaFree(d_seq);
  cudaFree(d_E);
  cudaFree(d_err);
  return st == LABS_OK ? E : (int64_t)st;
}

extern "C" labs_status labs_energy_batch(const int8_t *seqs, int32_t n, int32_t L, int64_t *E_out, void *stream,
                                         int32_t check) {
  if (!seqs || !E_out || n < 0 || L < 1 || L > 65536) return LABS_EINVAL;
  if (n == 0) return LABS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  labs_status st = LABS_OK;
  int32_t *d_err = nullptr;
  int32_t err = 0;
  LABS_CU(cudaMallocAsync(&d_err, sizeof(int32_t), s));
  LABS_CU(cudaMemsetAsync(d_err, 0, sizeof(int32_t), s));
  LABS_CU(launch_energy(seqs, n, L, E_out, d_err, s));
  if (check) {
    LABS_CU(cudaMemcpyAsync(&err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LABS_CU(cudaStreamSynchronize(s));
    if (err) st = LABS_EINVAL;
  }
done:
  if (d_err) cudaFreeAsync(d_err, s);
  return st;
}

// Table 1's encoding (Section 4.2): the free half s_1..s_D as D binary
// digits, s_1 the most significant, +1 -> 0 and -1 -> 1, printed in
// hexadecimal with ceil(D/4) digits; the other half follows from Eq. 2.
static int hex_digit_value(char c) {
  if (c >= '0' && c <= '9') return c - '0';
  if (c >= 'a' && c <= 'f') return c - 'a' + 10;
  if (c >= 'A' && c <= 'F') return c - 'A' + 10;
  return -1;
}

extern "C" labs_status labs_from_hex(const char *hex, int32_t L, int8_t *seq_out) {
  if (!hex || !seq_out || L < LABS_L_MIN || L > LABS_L_MAX || !(L & 1)) return LABS_EINVAL;
  const int D = (L + 1) / 2;
  if (hex[0] == '0' && (hex[1] == 'x' || hex[1] == 'X')) hex += 2;
  const size_t n = std::strlen(hex);
  if (n == 0 || n > 4096) return LABS_EINVAL;
  // binary digits from the least significant: bit b of the code -> s_{D-b}
  std::vector<uint8_t> bits(std::max<size_t>(4 * n, (size_t)D), 0);
  for (size_t i = 0; i < n; ++i) {
    const int v = hex_digit_value(hex[n - 1 - i]);
    if (v < 0) return LABS_EINVAL;
    for (int k = 0; k < 4; ++k) bits[4 * i + k] = (uint8_t)((v >> k) & 1);
  }
  for (size_t b = (size_t)D; b < bits.size(); ++b)
    if (bits[b]) return LABS_EINVAL;  // more than D binary digits
  for (int i = 0; i < D; ++i) seq_out[i] = bits[(size_t)(D - 1 - i)] ? (int8_t)-1 : (int8_t)1;
  // Eq. 2 with 0-based indices: centre c = D-1, s[c+i] = (-1)^i s[c-i]
  const int c = D - 1;
  for (int i = 1; i <= c; ++i) seq_out[c + i] = (i & 1) ? (int8_t)-seq_out[c - i] : seq_out[c - i];
  return LABS_OK;
}

extern "C" labs_status labs_to_hex(const int8_t *seq, int32_t L, char *out, size_t out_len) {
  if (!seq || !out || L < LABS_L_MIN || L > LABS_L_MAX || !(L & 1)) return LABS_EINVAL;
  const int D = (L + 1) / 2, c = D - 1;
  const int digits = (D + 3) / 4;
  if (out_len < (size_t)digits + 1) return LABS_EINVAL;
  for (int i = 0; i < L; ++i)
    if (seq[i] != 1 && seq[i] != -1) return LABS_EINVAL;
  for (int i = 1; i <= c; ++i)
    if (seq[c + i] != ((i & 1) ? -seq[c - i] : seq[c - i])) return LABS_EINVAL;  // not skew-symmetric
  static const char kHex[] = "0123456789ABCDEF";
  // hex digit k (from the least significant) holds binary digits 4k..4k+3, binary digit b = [s_{D-b} = -1]
  for (int k = 0; k < digits; ++k) {
    int v = 0;
    for (int bit = 0; bit < 4; ++bit) {
      const int b = 4 * k + bit;
      if (b < D && seq[D - 1 - b] < 0) v |= 1 << bit;
    }
    out[digits - 1 - k] = kHex[v];
  }
  out[digits] = '\0';
  return LABS_OK;
}

static size_t workspace_size(int32_t space, int32_t L, int32_t n_seeds, int32_t walks_per_seed, int32_t walk_len) {
  // the argument rules of labs_walks
  if (!valid_space_L(space, L) || n_seeds < 1 || walks_per_seed < 1 || walk_len < 1 || walk_len > (1 << 26) ||
      (uint64_t)n_seeds * (uint64_t)walks_per_seed > (1ull << 31))
    return 0;
  const size_t n_walks = (size_t)n_seeds * (size_t)walks_per_seed;
  const size_t tb = (size_t)table_cap(walk_len) * key_words64(key_bits(space, L)) * 8;
  Buffers b;
  const size_t fixed = carve(b, nullptr, L, n_seeds, n_walks, 0, tb);
  if (tb > (SIZE_MAX - fixed) / n_walks) return SIZE_MAX;  // not representable: more than any device holds
  return carve(b, nullptr, L, n_seeds, n_walks, n_walks, tb);
}

extern "C" size_t labs_walks_workspace_size(int32_t L, int32_t n_seeds, int32_t walks_per_seed, int32_t walk_len) {
  return workspace_size(kSpaceSkew, L, n_seeds, walks_per_seed, walk_len);
}

extern "C" size_t labs_walks_full_workspace_size(int32_t L, int32_t n_seeds, int32_t walks_per_seed,
                                                 int32_t walk_len) {
  return workspace_size(kSpaceFull, L, n_seeds, walks_per_seed, walk_len);
}

namespace psaw {
namespace {

// Shared driver of labs_walks and labs_saw_round.
struct Run {
  RunConfig cfg;
  cudaStream_t s = 0;
  void *ws = nullptr;
  bool own_ws = false;
  Buffers b{};
  size_t n_walks = 0, g_chunk = 0, table_bytes = 0;
  uint32_t cap = 0;
  int kw64 = 0, W = 0;
  int launches = 0, walk_launches = 0;
  double walk_ms = 0.0;
  Timer timer;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> walk_ev;

  labs_status setup(void *user_ws, size_t user_bytes) {
    W = space_lag_words(cfg.space, cfg.L);
    cap = table_cap(cfg.walk_len);
    kw64 = key_words64(key_bits(cfg.space, cfg.L));
    table_bytes = (size_t)cap * kw64 * 8;
    n_walks = (size_t)cfg.n_seeds * (size_t)cfg.walks;
    const size_t fixed = carve(b, nullptr, cfg.L, cfg.n_seeds, n_walks, 0, table_bytes);
    if (user_ws) {
      if (user_bytes < fixed + table_bytes) return LABS_ENOMEM;
      g_chunk = std::min(n_walks, (user_bytes - fixed) / table_bytes);
      if (g_chunk < n_walks && g_chunk > 32) g_chunk = g_chunk / 32 * 32;
      ws = user_ws;
    } else {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return LABS_ECUDA;
      const size_t budget = free_b / 10 * 9;
      if (budget < fixed + table_bytes) return LABS_ENOMEM;
      g_chunk = std::min(n_walks, (budget - fixed) / table_bytes);
      if (g_chunk < n_walks && g_chunk > 32) g_chunk = g_chunk / 32 * 32;
      const size_t bytes = carve(b, nullptr, cfg.L, cfg.n_seeds, n_walks, g_chunk, table_bytes);
      retain_pool_memory();
      if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) return LABS_ENOMEM;
      own_ws = true;
    }
    carve(b, ws, cfg.L, cfg.n_seeds, n_walks, g_chunk, table_bytes);
    return LABS_OK;
  }

  WalkParams params(uint32_t round, uint32_t g_begin, uint32_t g_count) const {
    WalkParams p{};
    p.L = cfg.L;
    p.walk_len = cfg.walk_len;
    p.walks_per_problem = cfg.walks;
    p.n_problems = cfg.n_seeds;
    p.round = round;
    p.g_begin = g_begin;
    p.g_count = g_count;
    p.cap = cap;
    p.kw64 = kw64;
    p.recheck_every = cfg.recheck_every;
    p.seeds = b.seeds;
    p.done = b.done;
    p.tables = b.tables;
    p.w_bestE = b.w_bestE;
    p.w_moves = b.w_moves;
    p.w_stuck = b.w_stuck;
    p.w_best_step = b.w_best_step;
    p.w_key = b.w_key;
    p.p_evals = b.p_evals;
    p.p_round_best = b.p_round_best;
    p.err = b.err;
    p.plane_steps = b.plane_steps;
    p.variant = resolve_variant(cfg.kernel);
    p.space = cfg.space;
    set_muls(p);
    return p;
  }

  // Resolve labs_opts.kernel == 0 (see g_variant).  Runs before the problems'
  // state is initialised: the sample rounds write only per-walk outputs, the
  // tables and accumulators that the real rounds reset.
  labs_status pick_variant() {
    if (cfg.kernel != 0) return LABS_OK;
    if (cfg.space != kSpaceSkew) {
      cfg.kernel = kVariantFullScan;
      return LABS_OK;
    }
    const std::pair<int, int> key{W, ilog2(g_chunk)};
    {
      std::lock_guard<std::mutex> lock(g_variant_mu);
      auto it = g_variant.find(key);
      if (it != g_variant.end()) {
        cfg.kernel = it->second;
        return LABS_OK;
      }
    }
    // one CTA per walk is timed only for launches of at most kCtaMaxWalksPerSm
    // walks per SM: with more, one warp per walk already keeps the SMs busy and
    // the CTA's extra per-step work (every warp applies the move) only costs
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return LABS_ECUDA;
    const bool offer_cta = g_chunk <= (size_t)kCtaMaxWalksPerSm * (size_t)sms;
    const int32_t cand[3] = {kVariantFullScan, kVariantWarp, kVariantCta};
    float best_ms = 1e30f;
    int32_t best = kVariantFullScan;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LABS_ECUDA;
    labs_status st = LABS_OK;
    for (int32_t v : cand) {
      if (v == kVariantCta && !offer_cta) continue;
      WalkParams p = params(0xFFFFF000u, 0, (uint32_t)g_chunk);
      p.variant = v;
      p.walk_len = std::min(cfg.walk_len, kSampleSteps);  // the call's tables hold this many
      p.cap = visited_table_cap(p.walk_len);
      p.done = nullptr;
      p.recheck_every = 0;
      p.plane_steps = nullptr;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && st == LABS_OK; ++rep) {  // the first launch warms up
        if (cudaEventRecord(e0, s) != cudaSuccess || launch_walk_round(W, p, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          st = LABS_ECUDA;
      }
      if (st != LABS_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LABS_OK) return st;
    cfg.kernel = best;
    // a choice made on walks shorter than kSampleSteps holds for this call
    // only: their start-up (tables, first pivot) weighs more than in longer
    // walks, and the cached choice is meant for the step loop's rate
    if (cfg.walk_len >= kSampleSteps) {
      std::lock_guard<std::mutex> lock(g_variant_mu);
      g_variant[key] = best;
    }
    return LABS_OK;
  }

  cudaError_t launch_round(uint32_t round, int32_t *trace, uint32_t trace_begin, uint32_t trace_count) {
    for (size_t g0 = 0; g0 < n_walks; g0 += g_chunk) {
      WalkParams p = params(round, (uint32_t)g0, (uint32_t)std::min(g_chunk, n_walks - g0));
      p.trace_flips = trace;
      p.trace_begin = trace_begin;
      p.trace_count = trace ? trace_count : 0;
      cudaEvent_t e0 = timer.rec(s);
      cudaError_t e = launch_walk_round(W, p, s);
      cudaEvent_t e1 = timer.rec(s);
      if (e != cudaSuccess) return e;
      walk_ev.push_back({e0, e1});
      ++launches;
      ++walk_launches;
    }
    FinalizeParams f{};
    f.n_problems = cfg.n_seeds;
    f.walks_per_problem = cfg.walks;
    f.round = round;
    f.done = b.done;
    f.budget = b.budget;
    f.target = b.target;
    f.w_key = b.w_key;
    f.p_evals = b.p_evals;
    f.p_round_best = b.p_round_best;
    f.p_bestE = b.p_bestE;
    f.p_key = b.p_key;
    f.p_rounds = b.p_rounds;
    f.p_best_round = b.p_best_round;
    f.p_best_walk = b.p_best_walk;
    ++launches;
    return launch_finalize(f, s);
  }

  cudaError_t init_problems(const uint64_t *seeds_src, cudaMemcpyKind kind) {
    std::vector<uint64_t> bud(cfg.n_seeds, cfg.budget);
    std::vector<int64_t> tgt(cfg.n_seeds, cfg.target);
    cudaError_t e = cudaMemcpyAsync(b.seeds, seeds_src, sizeof(uint64_t) * cfg.n_seeds, kind, s);
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.budget, bud.data(), sizeof(uint64_t) * cfg.n_seeds, h2d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.target, tgt.data(), sizeof(int64_t) * cfg.n_seeds, h2d, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.plane_steps, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      ++launches;
      e = launch_init_problems(cfg.n_seeds, b.p_bestE, b.p_evals, b.p_round_best, b.done, b.p_rounds,
                               b.p_best_round, b.p_best_walk, b.p_key, s);
    }
    // pageable copies above complete before returning; keep host vectors alive until then
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  }

  labs_status error_status() {
    int32_t err = 0;
    if (cudaMemcpyAsync(&err, b.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LABS_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LABS_ECUDA;
    if (err & kErrOverflow) return LABS_EOVERFLOW;
    if (err & kErrRecheck) return LABS_ECHECK;
    return LABS_OK;
  }

  void finish_timing() {
    for (auto &pr : walk_ev) walk_ms += elapsed(pr.first, pr.second);
  }

  ~Run() {
    if (own_ws && ws) cudaFreeAsync(ws, s);
  }
};

}  // namespace
}  // namespace psaw

static labs_status walks_impl(int32_t space, int32_t L, const uint64_t *seeds, int32_t n_seeds,
                              int32_t walks_per_seed, int32_t walk_len, uint64_t step_budget, int8_t *best_seq,
                              int64_t *best_E, const labs_opts *opts_in, labs_stats *stats) {
  labs_opts opts;
  if (opts_in) opts = *opts_in;
  else labs_opts_init(&opts);
  // the full search space has the full-scan kernel only
  const int32_t max_kernel = space == kSpaceFull ? kVariantFullScan : kVariantCta;
  if (!valid_space_L(space, L) || !seeds || !best_seq || !best_E || n_seeds < 1 || walks_per_seed < 1 ||
      walk_len < 1 || walk_len > (1 << 26) || step_budget < 1 || opts.recheck_every < 0 || opts.max_rounds < 0 ||
      opts.kernel < 0 || opts.kernel > max_kernel)
    return LABS_EINVAL;
  if ((uint64_t)n_seeds * (uint64_t)walks_per_seed > (1ull << 31)) return LABS_EINVAL;
  labs_status st = LABS_OK;
  Run run;
  run.cfg = RunConfig{L, n_seeds, walks_per_seed, walk_len, opts.recheck_every, step_budget, opts.target_E,
                      opts.max_rounds, opts.kernel, space};
  run.s = (cudaStream_t)opts.stream;
  const cudaMemcpyKind in_kind = opts.device_buffers ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind out_kind = opts.device_buffers ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const uint64_t full_round = (uint64_t)walks_per_seed * (uint64_t)walk_len * (uint64_t)key_bits(space, L);
  uint64_t est = (step_budget + full_round - 1) / full_round;
  if (opts.max_rounds > 0) est = std::min<uint64_t>(est, (uint64_t)opts.max_rounds);
  uint32_t round = 0;
  std::vector<int32_t> done_h(n_seeds);
  cudaEvent_t t0 = nullptr, t1 = nullptr;

  st = run.setup(opts.workspace, opts.workspace_bytes);
  if (st != LABS_OK) return st;
  if ((st = run.pick_variant()) != LABS_OK) return st;
  LABS_CU(run.init_problems(seeds, in_kind));
  t0 = run.timer.rec(run.s);
  for (;;) {
    // rounds are enqueued speculatively (a finished problem's later rounds are
    // no-ops on the device), at most kRoundBatch before the host looks again
    const uint32_t stop = (uint32_t)std::min<uint64_t>(est, (uint64_t)round + kRoundBatch);
    for (; round < stop; ++round) LABS_CU(run.launch_round(round, nullptr, 0, 0));
    LABS_CU(cudaMemcpyAsync(done_h.data(), run.b.done, sizeof(int32_t) * n_seeds, cudaMemcpyDeviceToHost, run.s));
    LABS_CU(cudaStreamSynchronize(run.s));
    bool all = true;
    for (int i = 0; i < n_seeds; ++i) all = all && done_h[i];
    if (all || (opts.max_rounds > 0 && round >= (uint32_t)opts.max_rounds)) break;
    if (round >= est) est = round + 1;
  }
  ++run.launches;
  LABS_CU(launch_expand(n_seeds, L, run.b.p_key, kKeyWords, run.b.best_seq, run.s, space == kSpaceFull));
  t1 = run.timer.rec(run.s);
  LABS_CU(cudaMemcpyAsync(best_seq, run.b.best_seq, (size_t)n_seeds * L, out_kind, run.s));
  LABS_CU(cudaMemcpyAsync(best_E, run.b.p_bestE, sizeof(int64_t) * n_seeds, out_kind, run.s));
  if (opts.evals_per_seed)
    LABS_CU(cudaMemcpyAsync(opts.evals_per_seed, run.b.p_evals, sizeof(uint64_t) * n_seeds, out_kind, run.s));
  if (opts.rounds_per_seed)
    LABS_CU(cudaMemcpyAsync(opts.rounds_per_seed, run.b.p_rounds, sizeof(int32_t) * n_seeds, out_kind, run.s));
  st = run.error_status();
  if (st != LABS_OK) goto done;
  if (stats) {
    std::vector<unsigned long long> ev(n_seeds);
    std::vector<int32_t> rounds(n_seeds);
    unsigned long long planes = 0;
    LABS_CU(cudaMemcpyAsync(&planes, run.b.plane_steps, sizeof(planes), cudaMemcpyDeviceToHost, run.s));
    LABS_CU(cudaMemcpyAsync(ev.data(), run.b.p_evals, sizeof(uint64_t) * n_seeds, cudaMemcpyDeviceToHost, run.s));
    LABS_CU(cudaMemcpyAsync(rounds.data(), run.b.p_rounds, sizeof(int32_t) * n_seeds, cudaMemcpyDeviceToHost, run.s));
    LABS_CU(cudaStreamSynchronize(run.s));
    run.finish_timing();
    std::memset(stats, 0, sizeof(*stats));
    for (int i = 0; i < n_seeds; ++i) {
      stats->evals += ev[i];
      stats->rounds = std::max(stats->rounds, rounds[i]);
    }
    stats->launches = run.launches;
    stats->walk_launches = run.walk_launches;
    stats->walk_kernel_ms = run.walk_ms;
    stats->device_ms = elapsed(t0, t1);
    stats->plane_steps = planes;
  }
done:
  if (st == LABS_OK) {
    cudaError_t e = cudaStreamSynchronize(run.s);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  return st;
}

extern "C" labs_status labs_walks(int32_t L, const uint64_t *seeds, int32_t n_seeds, int32_t walks_per_seed,
                                  int32_t walk_len, uint64_t step_budget, int8_t *best_seq, int64_t *best_E,
                                  const labs_opts *opts, labs_stats *stats) {
  return walks_impl(kSpaceSkew, L, seeds, n_seeds, walks_per_seed, walk_len, step_budget, best_seq, best_E, opts,
                    stats);
}

extern "C" labs_status labs_walks_full(int32_t L, const uint64_t *seeds, int32_t n_seeds, int32_t walks_per_seed,
                                       int32_t walk_len, uint64_t step_budget, int8_t *best_seq, int64_t *best_E,
                                       const labs_opts *opts, labs_stats *stats) {
  return walks_impl(kSpaceFull, L, seeds, n_seeds, walks_per_seed, walk_len, step_budget, best_seq, best_E, opts,
                    stats);
}

static labs_status saw_round_impl(int32_t space, int32_t L, uint64_t seed, uint32_t round, int32_t n_walks,
                                  int32_t walk_len, int32_t recheck_every, int64_t *walk_best_E,
                                  int8_t *walk_best_seq, int32_t *walk_moves, int32_t *walk_stuck,
                                  int32_t *walk_best_step, int32_t *trace_flips, int32_t trace_begin,
                                  int32_t trace_count, int32_t visited_walk, uint64_t *visited_keys,
                                  int32_t visited_cap, int32_t *visited_count, int32_t kernel) {
  const int32_t max_kernel = space == kSpaceFull ? kVariantFullScan : kVariantCta;
  if (!valid_space_L(space, L) || n_walks < 1 || walk_len < 1 || walk_len > (1 << 26) || recheck_every < 0 ||
      kernel < 0 || kernel > max_kernel)
    return LABS_EINVAL;
  if (trace_flips && (trace_begin < 0 || trace_count < 0 || (int64_t)trace_begin + trace_count > n_walks))
    return LABS_EINVAL;
  if (visited_keys && (visited_walk < 0 || visited_walk >= n_walks || visited_cap < 0 || !visited_count))
    return LABS_EINVAL;
  const int D = key_bits(space, L);
  labs_status st = LABS_OK;
  Run run;
  run.cfg = RunConfig{L, 1, n_walks, walk_len, recheck_every, ~0ull, -1, 1, kernel, space};
  run.s = 0;
  int32_t *d_trace = nullptr;
  int8_t *d_seqs = nullptr;
  std::vector<int32_t> i32(n_walks);
  const size_t trace_n = trace_flips ? (size_t)trace_count * (size_t)walk_len : 0;

  st = run.setup(nullptr, 0);
  if (st != LABS_OK) return st;
  if (run.g_chunk < (size_t)n_walks) return LABS_ENOMEM;  // the tables of the round must stay resident
  if ((st = run.pick_variant()) != LABS_OK) return st;
  LABS_CU(run.init_problems(&seed, cudaMemcpyHostToDevice));
  if (trace_n) {
    LABS_CU(cudaMalloc(&d_trace, trace_n * sizeof(int32_t)));
    LABS_CU(cudaMemset(d_trace, 0xFF, trace_n * sizeof(int32_t)));
  }
  LABS_CU(run.launch_round(round, d_trace, (uint32_t)trace_begin, (uint32_t)trace_count));
  st = run.error_status();
  if (st != LABS_OK) goto done;
  if (walk_best_E) {
    LABS_CU(cudaMemcpy(i32.data(), run.b.w_bestE, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n_walks; ++i) walk_best_E[i] = i32[i];
  }
  if (walk_moves) LABS_CU(cudaMemcpy(walk_moves, run.b.w_moves, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToHost));
  if (walk_stuck) LABS_CU(cudaMemcpy(walk_stuck, run.b.w_stuck, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToHost));
  if (walk_best_step)
    LABS_CU(cudaMemcpy(walk_best_step, run.b.w_best_step, sizeof(int32_t) * n_walks, cudaMemcpyDeviceToHost));
  if (walk_best_seq) {
    LABS_CU(cudaMalloc(&d_seqs, (size_t)n_walks * L));
    LABS_CU(launch_expand(n_walks, L, run.b.w_key, kKeyWords, d_seqs, 0, space == kSpaceFull));
    LABS_CU(cudaMemcpy(walk_best_seq, d_seqs, (size_t)n_walks * L, cudaMemcpyDeviceToHost));
  }
  if (trace_n) LABS_CU(cudaMemcpy(trace_flips, d_trace, trace_n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (visited_keys) {
    const size_t words = run.table_bytes / 8;
    std::vector<uint64_t> tbl(words);
    LABS_CU(cudaMemcpy(tbl.data(), run.b.tables + (size_t)visited_walk * words, run.table_bytes,
                       cudaMemcpyDeviceToHost));
    const int kout = (D + 63) / 64;
    int32_t cnt = 0;
    for (uint32_t sl = 0; sl < run.cap; ++sl) {
      const uint64_t *e = tbl.data() + (size_t)sl * run.kw64;
      bool empty = true;
      for (int i = 0; i < run.kw64; ++i) empty = empty && e[i] == 0;
      if (empty) continue;
      if (cnt < visited_cap) {
        for (int i = 0; i < kout; ++i) {
          uint64_t v = e[i];
          if ((D >> 6) == i) v &= ~(1ull << (D & 63));  // drop the occupancy flag
          visited_keys[(size_t)cnt * kout + i] = v;
        }
      }
      ++cnt;
    }
    *visited_count = cnt;
  }
done:
  if (d_trace) cudaFree(d_trace);
  if (d_seqs) cudaFree(d_seqs);
  if (st == LABS_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_status(e);
  }
  return st;
}

extern "C" labs_status labs_saw_round(int32_t L, uint64_t seed, uint32_t round, int32_t n_walks, int32_t walk_len,
                                      int32_t recheck_every, int64_t *walk_best_E, int8_t *walk_best_seq,
                                      int32_t *walk_moves, int32_t *walk_stuck, int32_t *walk_best_step,
                                      int32_t *trace_flips, int32_t trace_begin, int32_t trace_count,
                                      int32_t visited_walk, uint64_t *visited_keys, int32_t visited_cap,
                                      int32_t *visited_count, int32_t kernel) {
  return saw_round_impl(kSpaceSkew, L, seed, round, n_walks, walk_len, recheck_every, walk_best_E, walk_best_seq,
                        walk_moves, walk_stuck, walk_best_step, trace_flips, trace_begin, trace_count, visited_walk,
                        visited_keys, visited_cap, visited_count, kernel);
}

extern "C" labs_status labs_saw_round_full(int32_t L, uint64_t seed, uint32_t round, int32_t n_walks,
                                           int32_t walk_len, int32_t recheck_every, int64_t *walk_best_E,
                                           int8_t *walk_best_seq, int32_t *walk_moves, int32_t *walk_stuck,
                                           int32_t *walk_best_step, int32_t *trace_flips, int32_t trace_begin,
                                           int32_t trace_count, int32_t visited_walk, uint64_t *visited_keys,
                                           int32_t visited_cap, int32_t *visited_count) {
  return saw_round_impl(kSpaceFull, L, seed, round, n_walks, walk_len, recheck_every, walk_best_E, walk_best_seq,
                        walk_moves, walk_stuck, walk_best_step, trace_flips, trace_begin, trace_count, visited_walk,
                        visited_keys, visited_cap, visited_count, 0);
}
