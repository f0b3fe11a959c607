// Host side of the batched entry points (include/labs.h, labs_batch_*):
// many independent problems of uneven L solved together by the persistent
// batch kernel, launch after launch, with the launch sequence captured once as
// a CUDA graph when the plan is fixed in advance, and launch shapes (walks per
// CTA, visited-table capacity) chosen by timing candidates on a sample.
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
  int block = 128;
  int factor_x10 = 15;
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
std::map<TuneKey, std::pair<int, int>> g_tuned;  // -> (block, factor_x10)

int ilog2(uint64_t x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
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
  // device state
  BatchProblem *d_probs = nullptr;
  uint64_t *d_budget = nullptr;
  int64_t *d_target = nullptr;
  int32_t *d_done = nullptr, *d_best_round = nullptr, *d_best_walk = nullptr, *d_rounds = nullptr;
  int64_t *d_bestE = nullptr;
  uint32_t *d_key = nullptr;
  unsigned long long *d_evals = nullptr;
  int8_t *d_seq = nullptr;
  size_t seq_total = 0;
  std::vector<size_t> seq_off;
  // slots of the current launch
  size_t slots_cap = 0;
  uint32_t max_chunks = 1;
  unsigned long long *d_slot_best = nullptr, *d_slot_evals = nullptr;
  uint32_t *d_slot_keys = nullptr, *d_slot_round = nullptr;
  uint32_t *d_first_slot = nullptr, *d_n_slots = nullptr;
  unsigned int *d_task_next = nullptr;  // one counter per class
  unsigned long long *d_planes = nullptr;
  unsigned long long *d_rb_scratch = nullptr;  // per problem, for the state reset kernel
  int32_t *d_err = nullptr;
  // host mirrors of the last run
  std::vector<int64_t> h_bestE;
  std::vector<unsigned long long> h_evals;
  std::vector<int32_t> h_rounds, h_done;
  std::vector<int8_t> h_seq;
  bool have_results = false;
  // graph of the first launch plan (problems without targets)
  cudaGraphExec_t graph = nullptr;
  bool graph_plan_built = false;
  int launches_per_graph = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> graph_events;
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
  for (auto &pe : graph_events) {
    cudaEventDestroy(pe.first);
    cudaEventDestroy(pe.second);
  }
  for (auto &c : cls) {
    cudaFree(c.pool);
    cudaFree(c.tasks);
  }
  cudaFree(d_probs);
  cudaFree(d_budget);
  cudaFree(d_target);
  cudaFree(d_done);
  cudaFree(d_best_round);
  cudaFree(d_best_walk);
  cudaFree(d_rounds);
  cudaFree(d_bestE);
  cudaFree(d_key);
  cudaFree(d_evals);
  cudaFree(d_seq);
  cudaFree(d_slot_best);
  cudaFree(d_slot_evals);
  cudaFree(d_slot_keys);
  cudaFree(d_slot_round);
  cudaFree(d_first_slot);
  cudaFree(d_n_slots);
  cudaFree(d_task_next);
  cudaFree(d_planes);
  cudaFree(d_rb_scratch);
  cudaFree(d_err);
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

uint64_t full_round_evals(const labs_problem &p) {
  return (uint64_t)p.walks * (uint64_t)p.walk_len * (uint64_t)((p.L + 1) / 2);
}

// relative cost of one task (32 walks): steps x flips x lag words
double task_cost(const labs_problem &p) {
  const int D = (p.L + 1) / 2;
  return (double)p.walk_len * D * (double)lag_words(p.L);
}

BatchKernelParams kernel_params(labs_batch *b, ClassPlan &c, int ci) {
  BatchKernelParams k{};
  k.probs = b->d_probs;
  k.tasks = c.tasks;
  k.n_tasks = c.n_tasks;
  k.task_next = b->d_task_next + ci;
  k.pool = c.pool;
  k.pool_words = c.pool_words;
  k.slot_best = b->d_slot_best;
  k.slot_evals = b->d_slot_evals;
  k.slot_keys = b->d_slot_keys;
  k.max_chunks = b->max_chunks;
  k.done = b->d_done;
  k.mul_one = 1u;
  k.mul_two = 2u;
  k.mul_four = 4u;
  k.mul_h31 = 0x80000000u;
  k.mul_h30 = 0x40000000u;
  k.plane_steps = b->d_planes;
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
    c.resident = batch_resident_lanes(c.W, c.block);
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

labs_status ensure_slots(labs_batch *b, size_t n_slots) {
  if (n_slots <= b->slots_cap) return LABS_OK;
  cudaFree(b->d_slot_best);
  cudaFree(b->d_slot_evals);
  cudaFree(b->d_slot_keys);
  cudaFree(b->d_slot_round);
  b->slots_cap = std::max(n_slots, b->slots_cap * 2);
  BCU(dalloc(&b->d_slot_best, b->slots_cap));
  BCU(dalloc(&b->d_slot_evals, b->slots_cap));
  BCU(dalloc(&b->d_slot_keys, b->slots_cap * b->max_chunks * kKeyWords));
  BCU(dalloc(&b->d_slot_round, b->slots_cap));
  return LABS_OK;
}

// Plan one launch: rounds per problem (all the budget still needs, or at most
// rounds_per_launch for problems with a target), slots in round order, and
// each class's tasks sorted by decreasing cost (longest first).
labs_status plan_launch(labs_batch *b, const std::vector<int32_t> &next_round, const std::vector<int32_t> &done,
                        const std::vector<unsigned long long> &evals, size_t *n_slots_out) {
  const size_t n = b->pr.size();
  std::vector<uint32_t> first(n, 0), cnt(n, 0), slot_round;
  size_t slots = 0;
  for (size_t i = 0; i < n; ++i) {
    if (done[i]) continue;
    const labs_problem &p = b->pr[i];
    const uint64_t fr = full_round_evals(p);
    const uint64_t rem = p.step_budget > evals[i] ? p.step_budget - evals[i] : 0;
    uint64_t r = rem == 0 ? 1 : (rem + fr - 1) / fr;
    if (p.target_E >= 0) r = std::min<uint64_t>(r, (uint64_t)b->rounds_per_launch);
    r = std::max<uint64_t>(r, 1);
    first[i] = (uint32_t)slots;
    cnt[i] = (uint32_t)r;
    for (uint64_t k = 0; k < r; ++k) slot_round.push_back((uint32_t)(next_round[i] + k));
    slots += r;
  }
  labs_status st = ensure_slots(b, slots);
  if (st != LABS_OK) return st;
  for (size_t ci = 0; ci < b->cls.size(); ++ci) {
    ClassPlan &c = b->cls[ci];
    std::vector<std::pair<double, BatchTask>> tk;
    for (int i : c.probs) {
      if (done[i]) continue;
      const uint32_t chunks = (uint32_t)((b->pr[i].walks + 31) / 32);
      const double cost = task_cost(b->pr[i]);
      for (uint32_t k = 0; k < cnt[i]; ++k)
        for (uint32_t ch = 0; ch < chunks; ++ch)
          tk.push_back({cost, BatchTask{(uint32_t)i, slot_round[first[i] + k], ch, first[i] + k}});
    }
    using Costed = std::pair<double, BatchTask>;
    std::stable_sort(tk.begin(), tk.end(), [](const Costed &x, const Costed &y) {
      if (x.first != y.first) return x.first > y.first;
      return std::tie(x.second.round, x.second.problem, x.second.chunk) <
             std::tie(y.second.round, y.second.problem, y.second.chunk);
    });
    if (tk.size() > c.tasks_cap) {
      cudaFree(c.tasks);
      c.tasks_cap = std::max(tk.size(), 2 * c.tasks_cap);
      BCU(dalloc(&c.tasks, c.tasks_cap));
    }
    std::vector<BatchTask> flat(tk.size());
    for (size_t j = 0; j < tk.size(); ++j) flat[j] = tk[j].second;
    c.n_tasks = (uint32_t)flat.size();
    if (!flat.empty()) BCU(cudaMemcpy(c.tasks, flat.data(), sizeof(BatchTask) * flat.size(), cudaMemcpyHostToDevice));
  }
  if (slots) BCU(cudaMemcpy(b->d_slot_round, slot_round.data(), sizeof(uint32_t) * slots, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(b->d_first_slot, first.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(b->d_n_slots, cnt.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
  *n_slots_out = slots;
  return LABS_OK;
}

// Enqueue one planned launch: reset the slot accumulators and task counters,
// the persistent kernel of each class, then the in-order finalize.
labs_status enqueue_launch(labs_batch *b, size_t n_slots, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *ev,
                           int *launches) {
  if (n_slots) {
    BCU(cudaMemsetAsync(b->d_slot_best, 0xFF, sizeof(unsigned long long) * n_slots, b->s));
    BCU(cudaMemsetAsync(b->d_slot_evals, 0, sizeof(unsigned long long) * n_slots, b->s));
  }
  BCU(cudaMemsetAsync(b->d_task_next, 0, sizeof(unsigned int) * b->cls.size(), b->s));
  // fork: every class's kernel on its own stream after the resets, join before the finalize
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
      BCU(launch_batch(c.W, c.block, kernel_params(b, c, (int)ci), x, nullptr));
      ++*launches;
    }
    BCU(cudaEventRecord(b->cs_done[ci], x));
    BCU(cudaStreamWaitEvent(b->s, b->cs_done[ci], 0));
  }
  if (ev) {
    BCU(cudaEventRecord(e1, b->s));
    ev->push_back({e0, e1});
  }
  BatchFinalizeParams f{};
  f.n_problems = (int32_t)b->pr.size();
  f.first_slot = b->d_first_slot;
  f.n_slots = b->d_n_slots;
  f.slot_round = b->d_slot_round;
  f.slot_best = b->d_slot_best;
  f.slot_evals = b->d_slot_evals;
  f.slot_keys = b->d_slot_keys;
  f.max_chunks = b->max_chunks;
  f.budget = b->d_budget;
  f.target = b->d_target;
  f.done = b->d_done;
  f.bestE = b->d_bestE;
  f.key = b->d_key;
  f.best_round = b->d_best_round;
  f.best_walk = b->d_best_walk;
  f.evals = b->d_evals;
  f.rounds = b->d_rounds;
  BCU(launch_batch_finalize(f, b->s));
  ++*launches;
  return LABS_OK;
}

labs_status reset_state(labs_batch *b, int *launches) {
  const int n = (int)b->pr.size();
  BCU(launch_init_problems(n, b->d_bestE, b->d_evals, b->d_rb_scratch, b->d_done, b->d_rounds, b->d_best_round,
                           b->d_best_walk, b->d_key, b->s));
  BCU(cudaMemsetAsync(b->d_err, 0, sizeof(int32_t), b->s));
  BCU(cudaMemsetAsync(b->d_planes, 0, sizeof(unsigned long long), b->s));
  ++*launches;
  return LABS_OK;
}

labs_status expand_results(labs_batch *b, int *launches) {
  for (size_t i = 0; i < b->pr.size(); ++i) {
    BCU(launch_expand(1, b->pr[i].L, b->d_key + i * kKeyWords, kKeyWords, b->d_seq + b->seq_off[i], b->s));
    ++*launches;
  }
  return LABS_OK;
}

// Time candidate shapes (walks per CTA x table capacity) of one class on a
// sample of its round-0 tasks with walks shortened to at most 256 steps.
labs_status autotune_class(labs_batch *b, ClassPlan &c, int ci) {
  int max_len = 0, max_walks = 0;
  for (int i : c.probs) {
    max_len = std::max(max_len, b->pr[i].walk_len);
    max_walks = std::max(max_walks, b->pr[i].walks);
  }
  const TuneKey key{c.W, ilog2((uint64_t)max_len), ilog2((uint64_t)max_walks)};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      c.block = it->second.first;
      c.factor_x10 = it->second.second;
      return LABS_OK;
    }
  }
  const int blocks[] = {64, 128, 256};
  const int factors[] = {15, 30};
  float best_ms = 1e30f;
  int best_block = c.block, best_factor = c.factor_x10;
  // sample problems: the class's problems with short walks, round 0
  std::vector<labs_problem> saved = b->pr;
  for (int i : c.probs) b->pr[i].walk_len = std::min(b->pr[i].walk_len, 256);
  for (int fct : factors) {
    for (int blk : blocks) {
      c.block = blk;
      c.factor_x10 = fct;
      labs_status st = build_pools(b);
      if (st != LABS_OK) {
        b->pr = saved;
        return st;
      }
      // one wave of tasks
      std::vector<BatchTask> tk;
      const size_t want = (size_t)std::max(1, c.resident / 32);
      for (size_t k = 0; tk.size() < want && k < 4 * want; ++k) {
        const int i = c.probs[k % c.probs.size()];
        const uint32_t chunks = (uint32_t)((b->pr[i].walks + 31) / 32);
        tk.push_back(BatchTask{(uint32_t)i, 1000u + (uint32_t)(k / c.probs.size()), (uint32_t)(k % chunks), 0u});
      }
      st = ensure_slots(b, 1);
      if (st != LABS_OK) {
        b->pr = saved;
        return st;
      }
      if (tk.size() > c.tasks_cap) {
        cudaFree(c.tasks);
        c.tasks_cap = tk.size();
        if (dalloc(&c.tasks, c.tasks_cap) != cudaSuccess) {
          b->pr = saved;
          return LABS_ENOMEM;
        }
      }
      cudaMemcpy(c.tasks, tk.data(), sizeof(BatchTask) * tk.size(), cudaMemcpyHostToDevice);
      c.n_tasks = (uint32_t)tk.size();
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaMemsetAsync(b->d_task_next + ci, 0, sizeof(unsigned int), b->s);
        cudaMemsetAsync(b->d_slot_best, 0xFF, sizeof(unsigned long long), b->s);
        cudaEventRecord(e0, b->s);
        launch_batch(c.W, c.block, kernel_params(b, c, ci), b->s, nullptr);
        cudaEventRecord(e1, b->s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (cudaGetLastError() != cudaSuccess) {
        b->pr = saved;
        return LABS_ECUDA;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best_block = blk;
        best_factor = fct;
      }
    }
  }
  b->pr = saved;
  c.block = best_block;
  c.factor_x10 = best_factor;
  c.n_tasks = 0;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = {best_block, best_factor};
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
      opts.rounds_per_launch < 0)
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
  for (int i = 0; i < n; ++i) {
    const int W = lag_words(problems[i].L);
    b->W.push_back(W);
    ClassPlan *cp = nullptr;
    for (auto &c : b->cls)
      if (c.W == W) cp = &c;
    if (!cp) {
      b->cls.push_back(ClassPlan{});
      cp = &b->cls.back();
      cp->W = W;
      cp->block = opts.block_threads ? opts.block_threads : 128;
      cp->factor_x10 = opts.table_factor_x10 ? opts.table_factor_x10 : 15;
    }
    cp->probs.push_back(i);
    b->max_chunks = std::max<uint32_t>(b->max_chunks, (uint32_t)((problems[i].walks + 31) / 32));
    b->seq_off.push_back(b->seq_total);
    b->seq_total += (size_t)problems[i].L;
  }
  std::sort(b->cls.begin(), b->cls.end(), [](const ClassPlan &x, const ClassPlan &y) { return x.W > y.W; });
  if (cu(dalloc(&b->d_probs, n)) || cu(dalloc(&b->d_budget, n)) || cu(dalloc(&b->d_target, n)) ||
      cu(dalloc(&b->d_done, n)) || cu(dalloc(&b->d_best_round, n)) || cu(dalloc(&b->d_best_walk, n)) ||
      cu(dalloc(&b->d_rounds, n)) || cu(dalloc(&b->d_bestE, n)) || cu(dalloc(&b->d_key, (size_t)n * kKeyWords)) ||
      cu(dalloc(&b->d_evals, n)) || cu(dalloc(&b->d_seq, b->seq_total)) || cu(dalloc(&b->d_first_slot, n)) ||
      cu(dalloc(&b->d_n_slots, n)) || cu(dalloc(&b->d_task_next, b->cls.size())) || cu(dalloc(&b->d_planes, 1)) ||
      cu(dalloc(&b->d_err, 1)) || cu(dalloc(&b->d_rb_scratch, n)))
    return fail(LABS_ENOMEM);
  if (cudaMemset(b->d_done, 0, sizeof(int32_t) * n) != cudaSuccess ||
      cudaMemset(b->d_err, 0, sizeof(int32_t)) != cudaSuccess ||
      cudaMemset(b->d_planes, 0, sizeof(unsigned long long)) != cudaSuccess)
    return fail(LABS_ECUDA);
  std::vector<uint64_t> bud(n);
  std::vector<int64_t> tgt(n);
  for (int i = 0; i < n; ++i) {
    bud[i] = problems[i].step_budget;
    tgt[i] = problems[i].target_E;
  }
  if (cudaMemcpy(b->d_budget, bud.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_target, tgt.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LABS_ECUDA);
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
      const bool fixed = opts.block_threads && opts.table_factor_x10;
      if (!fixed && (st = autotune_class(b, c, (int)ci)) != LABS_OK) return fail(st);
      if (opts.block_threads) c.block = opts.block_threads;
      if (opts.table_factor_x10) c.factor_x10 = opts.table_factor_x10;
    }
    if ((st = build_pools(b)) != LABS_OK) return fail(st);
  }
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
  labs_status st = LABS_OK;
  BCU(cudaEventCreate(&t0));
  BCU(cudaEventCreate(&t1));
  BCU(cudaEventRecord(t0, b->s));
  bool first = true, continued = false;
  for (;;) {
    if (first && b->use_graph && !any_target) {
      // the first launch's plan is the same for every run: capture it once
      if (!b->graph) {
        size_t n_slots = 0;
        if ((st = plan_launch(b, next_round, done, evals, &n_slots)) != LABS_OK) return st;
        cudaGraph_t g = nullptr;
        BCU(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
        int cl = 0;
        labs_status cst = reset_state(b, &cl);
        if (cst == LABS_OK) cst = enqueue_launch(b, n_slots, nullptr, &cl);
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
      BCU(cudaGraphLaunch(b->graph, b->s));
      launches += b->launches_per_graph;
      for (auto &c : b->cls) walk_launches += c.n_tasks ? 1 : 0;
    } else {
      size_t n_slots = 0;
      if ((st = plan_launch(b, next_round, done, evals, &n_slots)) != LABS_OK) return st;
      if (first && (st = reset_state(b, &launches)) != LABS_OK) return st;
      const int before = launches;
      if ((st = enqueue_launch(b, n_slots, &ev, &launches)) != LABS_OK) return st;
      walk_launches += launches - before - 1;  // the finalize is the one non-walk launch
      continued = continued || !first;
    }
    first = false;
    std::vector<int32_t> rounds(n);
    BCU(cudaMemcpyAsync(done.data(), b->d_done, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->s));
    BCU(cudaMemcpyAsync(rounds.data(), b->d_rounds, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->s));
    BCU(cudaMemcpyAsync(evals.data(), b->d_evals, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, b->s));
    BCU(cudaStreamSynchronize(b->s));
    bool all = true;
    for (size_t i = 0; i < n; ++i) {
      all = all && done[i];
      next_round[i] = rounds[i];
    }
    if (all) break;
  }
  if (continued && b->graph) {
    // later launches reused the plan buffers the graph reads: capture afresh next run
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if ((st = expand_results(b, &launches)) != LABS_OK) return st;
  BCU(cudaEventRecord(t1, b->s));
  int32_t err = 0;
  unsigned long long planes = 0;
  b->h_bestE.resize(n);
  b->h_rounds.resize(n);
  b->h_seq.resize(b->seq_total);
  BCU(cudaMemcpyAsync(&err, b->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, b->s));
  BCU(cudaMemcpyAsync(&planes, b->d_planes, sizeof(planes), cudaMemcpyDeviceToHost, b->s));
  BCU(cudaMemcpyAsync(b->h_bestE.data(), b->d_bestE, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, b->s));
  BCU(cudaMemcpyAsync(b->h_rounds.data(), b->d_rounds, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->s));
  BCU(cudaMemcpyAsync(b->h_seq.data(), b->d_seq, b->seq_total, cudaMemcpyDeviceToHost, b->s));
  BCU(cudaStreamSynchronize(b->s));
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
    for (size_t i = 0; i < n; ++i) {
      stats->evals += evals[i];
      stats->rounds = std::max(stats->rounds, b->h_rounds[i]);
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
  if (best_seq) std::memcpy(best_seq, b->h_seq.data() + b->seq_off[i], (size_t)b->pr[i].L);
  if (best_E) *best_E = b->h_bestE[i];
  if (evals) *evals = b->h_evals[i];
  if (rounds) *rounds = b->h_rounds[i];
  return LABS_OK;
}

extern "C" labs_status labs_batch_shape(const labs_batch *b, int32_t W, int32_t *block_threads,
                                        int32_t *table_factor_x10, int32_t *resident_walks) {
  if (!b) return LABS_EINVAL;
  for (auto &c : b->cls) {
    if (c.W != W) continue;
    if (block_threads) *block_threads = c.block;
    if (table_factor_x10) *table_factor_x10 = c.factor_x10;
    if (resident_walks) *resident_walks = c.resident;
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
