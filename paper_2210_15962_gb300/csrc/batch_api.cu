// Host side of the batched entry points (include/labs.h, labs_batch_*):
// many independent problems of uneven L solved together by the persistent
// batch kernel, launch after launch, with the first launch sequence captured
// once as a CUDA graph when the plan is fixed in advance, and launch shapes
// (walks per CTA, visited-table capacity) chosen by timing candidates on a
// sample.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/labs.h"
#include "batch.cuh"

namespace psaw {
namespace {

constexpr uint32_t kMaxRingRounds = 1024;  // rounds of one problem issued in one launch at most
// key slots of the autotuner's record: more than any one wave of tasks needs
// (warps resident on a 152-SM device, 64 per SM)
constexpr size_t kTuneKeySlots = 152 * 64;
// Warp mode (one walk per warp) keeps a key slot per walk in every round
// record, so it is offered only while every problem has at most this many walks.
constexpr int kWarpModeMaxWalks = 4096;

bool valid_problem(const labs_problem &p) {
  return p.L >= LABS_L_MIN && p.L <= LABS_L_MAX && (p.L & 1) && p.walks >= 1 && p.walks <= (1 << 24) &&
         p.walk_len >= 1 && p.walk_len <= (1 << 26) && p.step_budget >= 1;
}

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void **)p, n * sizeof(T));
}

struct ClassPlan {
  int W = 0;
  bool warp = false;  // warp mode: one walk per warp, tasks of one walk
  bool cta = false;   // CTA mode: one walk per CTA of 128 threads, tasks of one walk
  bool per_walk() const { return warp || cta; }
  int unroll = 1;     // lane mode: the scan's flip loop unrolled 1 or 2 times
  int block = 128;
  int factor_x10 = kTableFactorX10;
  std::vector<int> probs;  // problem indices of this class
  size_t pool_words = 0;
  int resident = 0;
  uint64_t *pool = nullptr;
  BatchTask *tasks = nullptr;
  size_t tasks_cap = 0;
  uint32_t n_tasks = 0;
};

struct TuneKey {
  int W, walk_len_log2, walks_log2;
  bool operator<(const TuneKey &o) const {
    return std::tie(W, walk_len_log2, walks_log2) < std::tie(o.W, o.walk_len_log2, o.walks_log2);
  }
};
std::mutex g_tune_mu;
struct Tuned {
  int block, factor_x10;
  bool warp, cta;
  int unroll;
};
std::map<TuneKey, Tuned> g_tuned;

int ilog2(uint64_t x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

uint64_t full_round_evals(const labs_problem &p) {
  return (uint64_t)p.walks * (uint64_t)p.walk_len * (uint64_t)((p.L + 1) / 2);
}

// Rounds a problem still needs for its budget, given the evaluations done.
uint64_t rounds_needed(const labs_problem &p, uint64_t evals_done) {
  const uint64_t fr = full_round_evals(p);
  const uint64_t rem = p.step_budget > evals_done ? p.step_budget - evals_done : 0;
  return std::max<uint64_t>(1, (rem + fr - 1) / fr);
}

}  // namespace
}  // namespace psaw

using namespace psaw;

struct labs_batch {
  std::vector<labs_problem> pr;
  std::vector<int> W;  // class of each problem
  std::vector<ClassPlan> cls;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  bool use_graph = false;
  int rounds_per_launch = 4;
  bool warp_allowed = false;  // every problem has at most kWarpModeMaxWalks walks
  // per-problem device state, one allocation
  void *state_block = nullptr;
  BatchProblem *d_probs = nullptr;
  ProblemState ps{};
  uint32_t *d_rec_base = nullptr, *d_ring = nullptr;
  int32_t *d_all = nullptr;  // 0 .. n-1
  std::vector<uint32_t> rec_base, ring;
  // round records (one ring per problem, plus one record the autotuner's sample uses)
  void *rec_block = nullptr;
  uint32_t *keys_block = nullptr;  // the records' key slots, sized once the classes' modes are known
  unsigned long long *d_key_base = nullptr;
  RoundRecords rec{};
  uint32_t n_records = 0, tune_record = 0;
  // per launch
  RecordInit *d_issue = nullptr;
  size_t issue_cap = 0;
  int n_issue = 0;
  unsigned int *d_task_next = nullptr;  // one counter per class
  int32_t *d_err = nullptr;
  // read back after every launch, one block: done, rounds, best E, evals, planes, sequences
  char *d_snap = nullptr;
  size_t snap_bytes = 0;
  Snapshot snap{};
  int seq_stride = 0;  // the largest L
  std::vector<char> h_snap;
  // host mirrors of the last run
  std::vector<int64_t> h_bestE;
  std::vector<unsigned long long> h_evals, h_planes;
  std::vector<int32_t> h_rounds, h_done;
  std::vector<int8_t> h_seq;
  bool have_results = false;
  // graph of the first launch plan (problems without targets)
  cudaGraphExec_t graph = nullptr;
  int launches_per_graph = 0;
  // one stream per class so the classes' persistent kernels overlap (each
  // class's tail runs beside the next class's work)
  std::vector<cudaStream_t> cs;
  std::vector<cudaEvent_t> cs_done;
  cudaEvent_t fork = nullptr;

  ~labs_batch();
};

labs_batch::~labs_batch() {
  if (graph) cudaGraphExecDestroy(graph);
  for (auto x : cs) cudaStreamDestroy(x);
  for (auto e : cs_done) cudaEventDestroy(e);
  if (fork) cudaEventDestroy(fork);
  for (auto &c : cls) {
    cudaFree(c.pool);
    cudaFree(c.tasks);
  }
  cudaFree(state_block);
  cudaFree(rec_block);
  cudaFree(keys_block);
  cudaFree(d_issue);
  cudaFree(d_task_next);
  cudaFree(d_err);
  cudaFree(d_snap);
  if (own_stream && s) cudaStreamDestroy(s);
}

namespace psaw {
namespace {

labs_status cu(cudaError_t e) {
  if (e == cudaSuccess) return LABS_OK;
  return e == cudaErrorMemoryAllocation ? LABS_ENOMEM : LABS_ECUDA;
}

#define BCU(call)                         \
  do {                                    \
    labs_status st_ = cu(call);           \
    if (st_ != LABS_OK) return st_;       \
  } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

double task_cost(const labs_problem &p) { return batch_task_cost(p.L, p.walk_len); }

BatchKernelParams kernel_params(labs_batch *b, ClassPlan &c, int ci) {
  BatchKernelParams k{};
  k.probs = b->d_probs;
  k.tasks = c.tasks;
  k.n_tasks = c.n_tasks;
  k.task_next = b->d_task_next + ci;
  k.pool = c.pool;
  k.pool_words = c.pool_words;
  k.rec = b->rec;
  k.ps = b->ps;
  k.mul_one = 1u;
  k.mul_two = 2u;
  k.mul_four = 4u;
  k.mul_h31 = 0x80000000u;
  k.mul_h30 = 0x40000000u;
  k.err = b->d_err;
  return k;
}

// (Re)build the per-class visited-table pools for the chosen shapes.
labs_status build_pools(labs_batch *b) {
  for (auto &c : b->cls) {
    cudaFree(c.pool);
    c.pool = nullptr;
    size_t words = 0;
    for (int i : c.probs) {
      const size_t w = (size_t)visited_table_cap(b->pr[i].walk_len, c.factor_x10) * key_words64((b->pr[i].L + 1) / 2);
      words = std::max(words, w);
    }
    c.pool_words = (words + 1) / 2 * 2;
    // a table per lane, or per warp in warp mode
    c.resident = c.cta    ? batch_resident_ctas(c.W)
                 : c.warp ? batch_resident_warps(c.W, c.block)
                          : batch_resident_lanes(c.W, c.block, c.unroll);
    if (c.resident <= 0) return LABS_ECUDA;
    BCU(dalloc(&c.pool, (size_t)c.resident * c.pool_words));
  }
  // caps depend on each class's factor
  std::vector<BatchProblem> hp(b->pr.size());
  for (size_t i = 0; i < b->pr.size(); ++i) {
    const labs_problem &p = b->pr[i];
    const ClassPlan *cp = nullptr;
    for (auto &c : b->cls)
      if (c.W == b->W[i]) cp = &c;
    hp[i].L = p.L;
    hp[i].W = b->W[i];
    hp[i].walk_len = p.walk_len;
    hp[i].walks = p.walks;
    hp[i].cap = visited_table_cap(p.walk_len, cp->factor_x10);
    hp[i].kw64 = key_words64((p.L + 1) / 2);
    hp[i].seed = p.seed;
  }
  BCU(cudaMemcpy(b->d_probs, hp.data(), sizeof(BatchProblem) * hp.size(), cudaMemcpyHostToDevice));
  return LABS_OK;
}

// Plan one launch from the host's view of each problem (done, rounds
// finalized, evaluations): the rounds each unfinished problem runs (what its
// budget still needs, at most its ring, and at most rounds_per_launch for a
// problem with a target), their records, and each class's tasks in launch
// order (order_tasks).
labs_status plan_launch(labs_batch *b, const std::vector<int32_t> &next_round, const std::vector<int32_t> &done,
                        const std::vector<unsigned long long> &evals) {
  const size_t n = b->pr.size();
  std::vector<RecordInit> issue;
  std::vector<std::vector<PlannedTask>> tk(b->cls.size());
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    for (int i : b->cls[ci].probs) {
      if (done[i]) continue;
      const labs_problem &p = b->pr[i];
      uint64_t r = std::min<uint64_t>(rounds_needed(p, evals[i]), b->ring[i]);
      if (p.target_E >= 0) r = std::min<uint64_t>(r, (uint64_t)b->rounds_per_launch);
      const bool per_walk = b->cls[ci].per_walk();
      const uint32_t chunks = per_walk ? (uint32_t)p.walks : (uint32_t)((p.walks + 31) / 32);
      const double cost = task_cost(p);
      for (uint32_t k = 0; k < (uint32_t)r; ++k) {
        const uint32_t round = (uint32_t)next_round[i] + k;
        const uint32_t rec = b->rec_base[i] + round % b->ring[i];
        issue.push_back(RecordInit{rec, round, chunks, per_walk ? 0u : 5u});
        for (uint32_t ch = 0; ch < chunks; ++ch)
          tk[ci].push_back({p.target_E >= 0 ? k : 0u, cost, BatchTask{(uint32_t)i, round, ch, rec}});
      }
    }
  }
  (void)n;
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    ClassPlan &c = b->cls[ci];
    order_tasks(tk[ci]);
    if (tk[ci].size() > c.tasks_cap) {
      cudaFree(c.tasks);
      c.tasks_cap = std::max(tk[ci].size(), 2 * c.tasks_cap);
      BCU(dalloc(&c.tasks, c.tasks_cap));
    }
    std::vector<BatchTask> flat(tk[ci].size());
    for (size_t j = 0; j < flat.size(); ++j) flat[j] = tk[ci][j].t;
    c.n_tasks = (uint32_t)flat.size();
    if (!flat.empty()) BCU(cudaMemcpy(c.tasks, flat.data(), sizeof(BatchTask) * flat.size(), cudaMemcpyHostToDevice));
  }
  if (issue.size() > b->issue_cap) {
    cudaFree(b->d_issue);
    b->issue_cap = std::max(issue.size(), 2 * b->issue_cap);
    BCU(dalloc(&b->d_issue, b->issue_cap));
  }
  b->n_issue = (int)issue.size();
  if (!issue.empty())
    BCU(cudaMemcpy(b->d_issue, issue.data(), sizeof(RecordInit) * issue.size(), cudaMemcpyHostToDevice));
  return LABS_OK;
}

// Enqueue one planned launch: the new rounds' records, the persistent kernel
// of each class on its own stream, the finalization of anything the kernels
// left, and the snapshot of every problem.
labs_status enqueue_launch(labs_batch *b, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *ev, int *launches) {
  const int n = (int)b->pr.size();
  BCU(launch_issue_records(b->d_issue, b->n_issue, b->rec, b->s));
  BCU(cudaMemsetAsync(b->d_task_next, 0, sizeof(unsigned int) * b->cls.size(), b->s));
  ++*launches;
  // fork: every class's kernel on its own stream, join before the finalize
  BCU(cudaEventRecord(b->fork, b->s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ev) {
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    BCU(cudaEventRecord(e0, b->s));
  }
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    ClassPlan &c = b->cls[ci];
    cudaStream_t x = b->cs[ci];
    BCU(cudaStreamWaitEvent(x, b->fork, 0));
    if (c.n_tasks) {
      if (c.cta) BCU(launch_batch_cta(c.W, kernel_params(b, c, (int)ci), x));
      else if (c.warp) BCU(launch_batch_warp(c.W, c.block, kernel_params(b, c, (int)ci), x));
      else BCU(launch_batch(c.W, c.block, kernel_params(b, c, (int)ci), x, nullptr, 0, c.unroll));
      ++*launches;
    }
    BCU(cudaEventRecord(b->cs_done[ci], x));
    BCU(cudaStreamWaitEvent(b->s, b->cs_done[ci], 0));
  }
  if (ev) {
    BCU(cudaEventRecord(e1, b->s));
    ev->push_back({e0, e1});
  }
  BCU(launch_batch_finalize(b->d_all, n, b->rec, b->ps, b->s));
  BCU(launch_snapshot(b->d_all, n, b->d_probs, b->ps, nullptr, 0, b->rec, b->snap, b->s));
  *launches += 2;
  return LABS_OK;
}

labs_status reset_state(labs_batch *b, int *launches) {
  BCU(launch_init_problems_state(b->d_all, (int)b->pr.size(), b->rec, b->ps, b->s));
  BCU(cudaMemsetAsync(b->d_err, 0, sizeof(int32_t), b->s));
  ++*launches;
  return LABS_OK;
}

// Rounds problem p's first launch runs.
uint32_t first_launch_rounds(const labs_batch *b, const labs_problem &p) {
  uint64_t r = std::min<uint64_t>(rounds_needed(p, 0), kMaxRingRounds);
  if (p.target_E >= 0) r = std::min<uint64_t>(r, (uint64_t)b->rounds_per_launch);
  return (uint32_t)r;
}

// Time candidate launch shapes of one class: lane mode (one walk per lane,
// tasks of 32 walks) with walks per CTA in {64, 128, 256}, table capacity in
// {1.5, 3} x pivots and the scan's flip loop unrolled once or twice, warp
// mode (one walk per warp) with 128 or 256 threads per CTA, and CTA mode (one
// walk per CTA of 128 threads).  Each candidate runs the class's first launch as far as one
// wave of its resident lanes (or warps) reaches, on rounds no solve uses, with
// walks shortened to at most 256 steps; the one with the lowest time per
// neighbour evaluation wins (cached per process).  The sample's tasks all
// count into one record that never completes.
labs_status autotune_class(labs_batch *b, ClassPlan &c, int ci) {
  int max_len = 0;
  uint64_t lane_tasks = 0, walk_tasks = 0;
  for (int i : c.probs) {
    const labs_problem &p = b->pr[i];
    max_len = std::max(max_len, p.walk_len);
    lane_tasks += (uint64_t)((p.walks + 31) / 32) * first_launch_rounds(b, p);
    walk_tasks += (uint64_t)p.walks * first_launch_rounds(b, p);
  }
  const TuneKey key{c.W, ilog2((uint64_t)max_len), ilog2(walk_tasks)};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      c.block = it->second.block;
      c.factor_x10 = it->second.factor_x10;
      c.warp = it->second.warp;
      c.cta = it->second.cta;
      c.unroll = it->second.unroll;
      return LABS_OK;
    }
  }
  struct Cand {
    bool warp, cta;
    int block, factor, unroll;
  };
  std::vector<Cand> cands;
  for (int u : {1, 2})
    for (int fct : {15, 30})
      for (int blk : {64, 128, 256}) cands.push_back({false, false, blk, fct, u});
  if (b->warp_allowed) {
    for (int blk : {128, 256}) cands.push_back({true, false, blk, kTableFactorX10, 1});
    cands.push_back({false, true, kWalkBlock, kTableFactorX10, 1});
  }
  double best_ns = 1e300;
  Cand best = {c.warp, c.cta, c.block, c.factor_x10, c.unroll};
  std::vector<labs_problem> saved = b->pr;
  for (int i : c.probs) b->pr[i].walk_len = std::min(b->pr[i].walk_len, 256);
  auto restore = [&](labs_status st) {
    b->pr = saved;
    return st;
  };
  for (const Cand &cd : cands) {
    c.warp = cd.warp;
    c.cta = cd.cta;
    c.block = cd.block;
    c.factor_x10 = cd.factor;
    c.unroll = cd.unroll;
    labs_status st = build_pools(b);
    if (st != LABS_OK) return restore(st);
    // the first launch's tasks, as far as one wave reaches
    const bool per_walk = cd.warp || cd.cta;
    const uint64_t wave = per_walk ? (uint64_t)c.resident : (uint64_t)c.resident / 32;
    const uint64_t want = std::max<uint64_t>(1, std::min(per_walk ? walk_tasks : lane_tasks, wave));
    std::vector<BatchTask> tk;
    for (uint64_t k = 0; tk.size() < want; ++k) {
      const int i = c.probs[k % c.probs.size()];
      const uint32_t units = per_walk ? (uint32_t)b->pr[i].walks : (uint32_t)((b->pr[i].walks + 31) / 32);
      const uint64_t pass = k / c.probs.size();
      tk.push_back(BatchTask{(uint32_t)i, 1000u + (uint32_t)(pass / units), (uint32_t)(pass % units),
                             b->tune_record});
    }
    if (tk.size() > c.tasks_cap) {
      cudaFree(c.tasks);
      c.tasks_cap = tk.size();
      if (dalloc(&c.tasks, c.tasks_cap) != cudaSuccess) return restore(LABS_ENOMEM);
    }
    if (cudaMemcpy(c.tasks, tk.data(), sizeof(BatchTask) * tk.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return restore(LABS_ECUDA);
    c.n_tasks = (uint32_t)tk.size();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    unsigned long long evals = 0;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
      cudaMemsetAsync(b->d_task_next + ci, 0, sizeof(unsigned int), b->s);
      cudaMemsetAsync(b->rec.left + b->tune_record, 0xFF, sizeof(uint32_t), b->s);
      cudaMemsetAsync(b->rec.evals + b->tune_record, 0, sizeof(unsigned long long), b->s);
      cudaEventRecord(e0, b->s);
      if (cd.cta) launch_batch_cta(c.W, kernel_params(b, c, ci), b->s);
      else if (cd.warp) launch_batch_warp(c.W, c.block, kernel_params(b, c, ci), b->s);
      else launch_batch(c.W, c.block, kernel_params(b, c, ci), b->s, nullptr, 0, c.unroll);
      cudaEventRecord(e1, b->s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaMemcpy(&evals, b->rec.evals + b->tune_record, sizeof(evals), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return restore(LABS_ECUDA);
    const double ns = 1e6 * (double)ms / (double)std::max<unsigned long long>(1, evals);
    if (ns < best_ns) {
      best_ns = ns;
      best = cd;
    }
  }
  b->pr = saved;
  c.warp = best.warp;
  c.cta = best.cta;
  c.block = best.block;
  c.factor_x10 = best.factor;
  c.unroll = best.unroll;
  c.n_tasks = 0;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = Tuned{best.block, best.factor, best.warp, best.cta, best.unroll};
  return LABS_OK;
}

// Device memory of the per-problem state, the round records and the snapshot.
labs_status alloc_state(labs_batch *b) {
  const size_t n = b->pr.size();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t o_probs = take(sizeof(BatchProblem) * n), o_budget = take(sizeof(uint64_t) * n),
               o_target = take(sizeof(int64_t) * n), o_base = take(sizeof(uint32_t) * n),
               o_ring = take(sizeof(uint32_t) * n), o_fin = take(sizeof(uint32_t) * n),
               o_done = take(sizeof(int32_t) * n), o_bestE = take(sizeof(int64_t) * n),
               o_key = take(sizeof(uint32_t) * kKeyWords * n), o_brnd = take(sizeof(int32_t) * n),
               o_bwalk = take(sizeof(int32_t) * n), o_evals = take(sizeof(unsigned long long) * n),
               o_planes = take(sizeof(unsigned long long) * n), o_rounds = take(sizeof(int32_t) * n),
               o_all = take(sizeof(int32_t) * n);
  char *sb = nullptr;
  BCU(cudaMalloc((void **)&sb, off));
  b->state_block = sb;
  b->d_probs = reinterpret_cast<BatchProblem *>(sb + o_probs);
  b->d_rec_base = reinterpret_cast<uint32_t *>(sb + o_base);
  b->d_ring = reinterpret_cast<uint32_t *>(sb + o_ring);
  b->d_all = reinterpret_cast<int32_t *>(sb + o_all);
  ProblemState &ps = b->ps;
  ps.rec_base = b->d_rec_base;
  ps.ring = b->d_ring;
  ps.budget = reinterpret_cast<uint64_t *>(sb + o_budget);
  ps.target = reinterpret_cast<int64_t *>(sb + o_target);
  ps.fin = reinterpret_cast<uint32_t *>(sb + o_fin);
  ps.done = reinterpret_cast<int32_t *>(sb + o_done);
  ps.bestE = reinterpret_cast<int64_t *>(sb + o_bestE);
  ps.key = reinterpret_cast<uint32_t *>(sb + o_key);
  ps.best_round = reinterpret_cast<int32_t *>(sb + o_brnd);
  ps.best_walk = reinterpret_cast<int32_t *>(sb + o_bwalk);
  ps.evals = reinterpret_cast<unsigned long long *>(sb + o_evals);
  ps.planes = reinterpret_cast<unsigned long long *>(sb + o_planes);
  ps.rounds = reinterpret_cast<int32_t *>(sb + o_rounds);
  std::vector<uint64_t> bud(n);
  std::vector<int64_t> tgt(n);
  std::vector<int32_t> all(n);
  for (size_t i = 0; i < n; ++i) {
    bud[i] = b->pr[i].step_budget;
    tgt[i] = b->pr[i].target_E;
    all[i] = (int32_t)i;
  }
  BCU(cudaMemset(sb, 0, off));
  BCU(cudaMemcpy(sb + o_budget, bud.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(sb + o_target, tgt.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(sb + o_base, b->rec_base.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(sb + o_ring, b->ring.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(sb + o_all, all.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  // records: the problems' rings and the autotuner's record
  const size_t nr = (size_t)b->n_records + 1;
  off = 0;
  const size_t r_best = take(sizeof(unsigned long long) * nr), r_evals = take(sizeof(unsigned long long) * nr),
               r_planes = take(sizeof(unsigned long long) * nr), r_left = take(sizeof(uint32_t) * nr),
               r_round = take(sizeof(uint32_t) * nr), r_shift = take(sizeof(uint32_t) * nr),
               r_kbase = take(sizeof(unsigned long long) * nr);
  char *rb = nullptr;
  BCU(cudaMalloc((void **)&rb, off));
  b->rec_block = rb;
  BCU(cudaMemset(rb, 0, off));
  BCU(cudaMemset(rb + r_round, 0xFF, sizeof(uint32_t) * nr));
  b->rec.best = reinterpret_cast<unsigned long long *>(rb + r_best);
  b->rec.evals = reinterpret_cast<unsigned long long *>(rb + r_evals);
  b->rec.planes = reinterpret_cast<unsigned long long *>(rb + r_planes);
  b->rec.left = reinterpret_cast<uint32_t *>(rb + r_left);
  b->rec.round = reinterpret_cast<uint32_t *>(rb + r_round);
  b->rec.shift = reinterpret_cast<uint32_t *>(rb + r_shift);
  b->d_key_base = reinterpret_cast<unsigned long long *>(rb + r_kbase);
  b->rec.key_base = b->d_key_base;
  b->tune_record = b->n_records;
  // until the classes' modes are known only the autotuner's record has key
  // slots (every record's base is 0 meanwhile; none of them runs before alloc_keys)
  BCU(dalloc(&b->keys_block, kTuneKeySlots * kKeyWords));
  b->rec.keys = b->keys_block;
  // the snapshot block
  off = 0;
  const size_t s_done = take(sizeof(int32_t) * n), s_rounds = take(sizeof(int32_t) * n),
               s_bestE = take(sizeof(int64_t) * n), s_evals = take(sizeof(unsigned long long) * n),
               s_planes = take(sizeof(unsigned long long) * n), s_seq = take(n * (size_t)b->seq_stride);
  BCU(cudaMalloc((void **)&b->d_snap, off));
  BCU(cudaMemset(b->d_snap, 0, off));
  b->snap_bytes = off;
  b->snap.done = reinterpret_cast<int32_t *>(b->d_snap + s_done);
  b->snap.rounds = reinterpret_cast<int32_t *>(b->d_snap + s_rounds);
  b->snap.bestE = reinterpret_cast<int64_t *>(b->d_snap + s_bestE);
  b->snap.evals = reinterpret_cast<unsigned long long *>(b->d_snap + s_evals);
  b->snap.planes = reinterpret_cast<unsigned long long *>(b->d_snap + s_planes);
  b->snap.seq = reinterpret_cast<int8_t *>(b->d_snap + s_seq);
  b->snap.stride = b->seq_stride;
  b->snap.run_evals = nullptr;
  b->h_snap.resize(off);
  BCU(dalloc(&b->d_task_next, b->cls.size()));
  BCU(dalloc(&b->d_err, 1));
  BCU(cudaMemset(b->d_err, 0, sizeof(int32_t)));
  return LABS_OK;
}

// Key slots of every record for the classes' chosen modes: a slot per chunk of
// 32 walks in lane mode, per walk in warp and CTA mode; the autotuner's slots first.
labs_status alloc_keys(labs_batch *b) {
  std::vector<unsigned long long> base(b->n_records + 1);
  unsigned long long next = kTuneKeySlots;
  base[b->tune_record] = 0;
  for (size_t i = 0; i < b->pr.size(); ++i) {
    bool per_walk = false;
    for (auto &c : b->cls)
      if (c.W == b->W[i]) per_walk = c.per_walk();
    const unsigned long long slots = per_walk ? (unsigned long long)b->pr[i].walks
                                              : (unsigned long long)((b->pr[i].walks + 31) / 32);
    for (uint32_t k = 0; k < b->ring[i]; ++k) {
      base[b->rec_base[i] + k] = next;
      next += slots;
    }
  }
  cudaFree(b->keys_block);
  b->keys_block = nullptr;
  BCU(dalloc(&b->keys_block, (size_t)next * kKeyWords));
  b->rec.keys = b->keys_block;
  BCU(cudaMemcpy(b->d_key_base, base.data(), sizeof(unsigned long long) * base.size(), cudaMemcpyHostToDevice));
  return LABS_OK;
}

// Copy the snapshot to the host (stream-ordered, then synchronised) and
// unpack the fields the run loop needs.
labs_status read_snapshot(labs_batch *b, std::vector<int32_t> &done, std::vector<int32_t> &rounds,
                          std::vector<unsigned long long> &evals) {
  BCU(cudaMemcpyAsync(b->h_snap.data(), b->d_snap, b->snap_bytes, cudaMemcpyDeviceToHost, b->s));
  BCU(cudaStreamSynchronize(b->s));
  const size_t n = b->pr.size();
  auto at = [&](const void *dev) { return b->h_snap.data() + ((const char *)dev - b->d_snap); };
  std::memcpy(done.data(), at(b->snap.done), sizeof(int32_t) * n);
  std::memcpy(rounds.data(), at(b->snap.rounds), sizeof(int32_t) * n);
  std::memcpy(evals.data(), at(b->snap.evals), sizeof(unsigned long long) * n);
  return LABS_OK;
}

}  // namespace
}  // namespace psaw

extern "C" labs_status labs_batch_create(const labs_problem *problems, int32_t n, const labs_batch_opts *opts_in,
                                         labs_batch **out) {
  if (!problems || n < 1 || !out) return LABS_EINVAL;
  *out = nullptr;
  labs_batch_opts opts;
  std::memset(&opts, 0, sizeof(opts));
  if (opts_in) opts = *opts_in;
  if (opts.block_threads < 0 || opts.block_threads > 256 || (opts.block_threads % 32) != 0 ||
      opts.table_factor_x10 < 0 || (opts.table_factor_x10 > 0 && opts.table_factor_x10 < 12) ||
      opts.rounds_per_launch < 0 || opts.rounds_per_launch > (int32_t)kMaxRingRounds || opts.walk_mode < 0 ||
      opts.walk_mode > 3)
    return LABS_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!valid_problem(problems[i])) return LABS_EINVAL;
  labs_batch *b = new (std::nothrow) labs_batch();
  if (!b) return LABS_ENOMEM;
  b->pr.assign(problems, problems + n);
  b->use_graph = opts.use_graph != 0;
  b->rounds_per_launch = opts.rounds_per_launch > 0 ? opts.rounds_per_launch : 4;
  if (opts.stream) {
    b->s = (cudaStream_t)opts.stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return LABS_ECUDA;
    }
    b->own_stream = true;
  }
  labs_status st = LABS_OK;
  auto fail = [&](labs_status e) {
    delete b;
    return e;
  };
  uint32_t max_walks = 1;
  for (int i = 0; i < n; ++i) {
    const labs_problem &p = problems[i];
    const int W = lag_words(p.L);
    b->W.push_back(W);
    ClassPlan *cp = nullptr;
    for (auto &c : b->cls)
      if (c.W == W) cp = &c;
    if (!cp) {
      b->cls.push_back(ClassPlan{});
      cp = &b->cls.back();
      cp->W = W;
      cp->block = opts.block_threads ? opts.block_threads : 128;
      cp->factor_x10 = opts.table_factor_x10 ? opts.table_factor_x10 : kTableFactorX10;
    }
    cp->probs.push_back(i);
    max_walks = std::max<uint32_t>(max_walks, (uint32_t)p.walks);
    b->seq_stride = std::max(b->seq_stride, (int)p.L);
    // the problem's ring: the rounds its first launch issues
    const uint32_t r = first_launch_rounds(b, p);
    b->rec_base.push_back(b->n_records);
    b->ring.push_back((uint32_t)r);
    b->n_records += (uint32_t)r;
  }
  b->warp_allowed = max_walks <= (uint32_t)kWarpModeMaxWalks && opts.walk_mode != 1;
  if (opts.walk_mode >= 2 && !b->warp_allowed) return fail(LABS_EINVAL);
  for (auto &c : b->cls) {
    c.warp = opts.walk_mode == 2;
    c.cta = opts.walk_mode == 3;
  }
  std::sort(b->cls.begin(), b->cls.end(), [](const ClassPlan &x, const ClassPlan &y) { return x.W > y.W; });
  if ((st = alloc_state(b)) != LABS_OK) return fail(st);
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    cudaStream_t x;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return fail(LABS_ECUDA);
    b->cs.push_back(x);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(LABS_ECUDA);
    b->cs_done.push_back(e);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return fail(LABS_ECUDA);
  if ((st = build_pools(b)) != LABS_OK) return fail(st);
  if (opts.autotune) {
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
      ClassPlan &c = b->cls[ci];
      const bool fixed = (opts.block_threads && opts.table_factor_x10) || opts.walk_mode >= 2;
      if (!fixed && (st = autotune_class(b, c, (int)ci)) != LABS_OK) return fail(st);
      if (opts.block_threads) c.block = opts.block_threads;
      if (opts.table_factor_x10) c.factor_x10 = opts.table_factor_x10;
    }
    if ((st = build_pools(b)) != LABS_OK) return fail(st);
  }
  if ((st = alloc_keys(b)) != LABS_OK) return fail(st);
  *out = b;
  return LABS_OK;
}

extern "C" labs_status labs_batch_run(labs_batch *b, labs_stats *stats) {
  if (!b) return LABS_EINVAL;
  const size_t n = b->pr.size();
  int launches = 0, walk_launches = 0;
  double walk_ms = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  std::vector<int32_t> next_round(n, 0), done(n, 0);
  std::vector<unsigned long long> evals(n, 0);
  bool any_target = false;
  for (auto &p : b->pr) any_target = any_target || p.target_E >= 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  BCU(cudaEventCreate(&t0));
  BCU(cudaEventCreate(&t1));
  BCU(cudaEventRecord(t0, b->s));
  bool first = true;
  for (;;) {
    if (first && b->use_graph && !any_target) {
      // the first launch's plan is the same for every run: capture it once
      if (!b->graph) {
        labs_status st = plan_launch(b, next_round, done, evals);
        if (st != LABS_OK) return st;
        cudaGraph_t g = nullptr;
        BCU(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
        int cl = 0;
        labs_status cst = reset_state(b, &cl);
        if (cst == LABS_OK) cst = enqueue_launch(b, nullptr, &cl);
        cudaError_t ee = cudaStreamEndCapture(b->s, &g);
        if (cst != LABS_OK) {
          if (g) cudaGraphDestroy(g);
          return cst;
        }
        BCU(ee);
        ee = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCU(ee);
        b->launches_per_graph = cl;
      }
      cudaEvent_t g0 = nullptr, g1 = nullptr;
      BCU(cudaEventCreate(&g0));
      BCU(cudaEventCreate(&g1));
      BCU(cudaEventRecord(g0, b->s));
      BCU(cudaGraphLaunch(b->graph, b->s));
      BCU(cudaEventRecord(g1, b->s));
      ev.push_back({g0, g1});
      launches += b->launches_per_graph;
      for (auto &c : b->cls) walk_launches += c.n_tasks ? 1 : 0;
    } else {
      labs_status st = plan_launch(b, next_round, done, evals);
      if (st != LABS_OK) return st;
      if (first && (st = reset_state(b, &launches)) != LABS_OK) return st;
      for (auto &c : b->cls) walk_launches += c.n_tasks ? 1 : 0;
      if ((st = enqueue_launch(b, &ev, &launches)) != LABS_OK) return st;
      if (!first && b->graph) {
        // the graph's task lists were replaced by this launch's: capture afresh next run
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
    }
    first = false;
    labs_status st = read_snapshot(b, done, next_round, evals);
    if (st != LABS_OK) return st;
    bool all = true;
    for (size_t i = 0; i < n; ++i) all = all && done[i];
    if (all) break;
  }
  BCU(cudaEventRecord(t1, b->s));
  int32_t err = 0;
  BCU(cudaMemcpyAsync(&err, b->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, b->s));
  BCU(cudaStreamSynchronize(b->s));
  auto at = [&](const void *dev) { return b->h_snap.data() + ((const char *)dev - b->d_snap); };
  b->h_bestE.resize(n);
  b->h_planes.resize(n);
  b->h_seq.resize(n * (size_t)b->seq_stride);
  std::memcpy(b->h_bestE.data(), at(b->snap.bestE), sizeof(int64_t) * n);
  std::memcpy(b->h_planes.data(), at(b->snap.planes), sizeof(unsigned long long) * n);
  std::memcpy(b->h_seq.data(), at(b->snap.seq), b->h_seq.size());
  b->h_rounds = next_round;
  b->h_evals = evals;
  b->h_done = done;
  b->have_results = true;
  for (auto &pe : ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.first, pe.second) == cudaSuccess) walk_ms += ms;
    cudaEventDestroy(pe.first);
    cudaEventDestroy(pe.second);
  }
  float dev_ms = 0.f;
  cudaEventElapsedTime(&dev_ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (err & kErrOverflow) return LABS_EOVERFLOW;
  if (err & kErrRecheck) return LABS_ECHECK;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    unsigned long long planes = 0;
    for (size_t i = 0; i < n; ++i) {
      stats->evals += evals[i];
      stats->rounds = std::max(stats->rounds, b->h_rounds[i]);
      planes += b->h_planes[i];
    }
    stats->launches = launches;
    stats->walk_launches = walk_launches;
    stats->walk_kernel_ms = walk_ms > 0 ? walk_ms : dev_ms;
    stats->device_ms = dev_ms;
    stats->plane_steps = planes;
  }
  return LABS_OK;
}

extern "C" labs_status labs_batch_result(const labs_batch *b, int32_t i, int8_t *best_seq, int64_t *best_E,
                                         uint64_t *evals, int32_t *rounds) {
  if (!b || i < 0 || (size_t)i >= b->pr.size()) return LABS_EINVAL;
  if (!b->have_results) return LABS_PENDING;
  if (best_seq) std::memcpy(best_seq, b->h_seq.data() + (size_t)i * b->seq_stride, (size_t)b->pr[i].L);
  if (best_E) *best_E = b->h_bestE[i];
  if (evals) *evals = b->h_evals[i];
  if (rounds) *rounds = b->h_rounds[i];
  return LABS_OK;
}

extern "C" labs_status labs_batch_plane_steps(const labs_batch *b, int32_t i, uint64_t *plane_steps) {
  if (!b || !plane_steps || i < 0 || (size_t)i >= b->pr.size()) return LABS_EINVAL;
  if (!b->have_results) return LABS_PENDING;
  *plane_steps = b->h_planes[i];
  return LABS_OK;
}

extern "C" labs_status labs_batch_shape(const labs_batch *b, int32_t W, int32_t *block_threads,
                                        int32_t *table_factor_x10, int32_t *resident_walks,
                                        int32_t *warp_per_walk, int32_t *unroll) {
  if (!b) return LABS_EINVAL;
  for (auto &c : b->cls) {
    if (c.W != W) continue;
    if (block_threads) *block_threads = c.cta ? kWalkBlock : c.block;  // a CTA-mode block is one walk's
    if (table_factor_x10) *table_factor_x10 = c.factor_x10;
    if (resident_walks) *resident_walks = c.resident;
    if (warp_per_walk) *warp_per_walk = c.cta ? 2 : (c.warp ? 1 : 0);
    if (unroll) *unroll = c.per_walk() ? 1 : c.unroll;
    return LABS_OK;
  }
  return LABS_ENOTFOUND;
}

extern "C" labs_status labs_batch_destroy(labs_batch *b) {
  if (!b) return LABS_EINVAL;
  cudaStreamSynchronize(b->s);
  delete b;
  return LABS_OK;
}
