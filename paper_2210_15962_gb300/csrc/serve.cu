// Serving loop with continuous batching (labs_serve_* in include/labs.h).
//
// Requests (one problem each) arrive at any time.  A scheduler thread admits
// them in arrival order into device slots while a slot is free and the
// server's memory budget holds their working set, then repeatedly launches
// the persistent batch kernels over every admitted request at once (a few
// rounds each per launch), finalizes each request round by round (Algorithm
// 1's best update and stop rule), hands finished requests back and admits
// newly arrived ones at the next launch boundary.  A request's result depends
// only on its own (L, seed, walks, walk_len, budget, target): the same alone
// and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/labs.h"
#include "batch.cuh"

namespace psaw {
namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket = 0;
  labs_problem p{};
  int W = 0;
  size_t mem_cost = 0;
  uint64_t t_submit = 0, t_admit = 0, t_done = 0;
  labs_status status = LABS_PENDING;
  int64_t bestE = -1;
  uint64_t evals = 0;
  int32_t rounds = 0;
  std::vector<int8_t> seq;
  int slot = -1;
  int32_t next_round = 0;
};

struct ClassPool {
  int W = 0;
  size_t words = 0;  // per lane
  int resident = 0;
  uint64_t *pool = nullptr;
  BatchTask *tasks = nullptr;
  size_t tasks_cap = 0;
  uint32_t n_tasks = 0;
};

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void **)p, (n ? n : 1) * sizeof(T));
}

}  // namespace
}  // namespace psaw

using namespace psaw;

struct labs_server {
  labs_serve_cfg cfg{};
  int device = 0;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  std::mutex mu;
  std::condition_variable wake;       // scheduler: new request or shutdown
  std::condition_variable finished;   // waiters: a request finished
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<uint64_t> slot_ticket;  // 0 = free
  size_t mem_used = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  labs_status failed = LABS_OK;
  std::thread th;
  // counters
  uint64_t n_submitted = 0, n_completed = 0, evals_done = 0, evals_run = 0;
  uint64_t launches = 0, walk_launches = 0;
  double busy_ms = 0.0;
  uint64_t t_created = 0;
  // device buffers, indexed by slot
  BatchProblem *d_probs = nullptr;
  uint64_t *d_budget = nullptr;
  int64_t *d_target = nullptr;
  int32_t *d_done = nullptr, *d_best_round = nullptr, *d_best_walk = nullptr, *d_rounds = nullptr;
  int64_t *d_bestE = nullptr;
  uint32_t *d_key = nullptr;
  unsigned long long *d_evals = nullptr;
  int32_t *d_init_list = nullptr;
  // per launch
  uint32_t max_chunks = 1, max_slots = 0;
  unsigned long long *d_slot_best = nullptr, *d_slot_evals = nullptr;
  uint32_t *d_slot_keys = nullptr, *d_slot_round = nullptr, *d_first_slot = nullptr, *d_n_slots = nullptr;
  unsigned int *d_task_next = nullptr;
  unsigned long long *d_planes = nullptr;
  int32_t *d_err = nullptr;
  int8_t *d_seq = nullptr;
  std::vector<ClassPool> pools;  // index W-1
  std::vector<cudaStream_t> cs;  // one stream per class (overlapping kernels)
  std::vector<cudaEvent_t> cs_done;
  cudaEvent_t fork = nullptr;

  ~labs_server();
  void loop();
  labs_status step(std::vector<int> &active);
};

labs_server::~labs_server() {
  for (auto x : cs) cudaStreamDestroy(x);
  for (auto e : cs_done) cudaEventDestroy(e);
  if (fork) cudaEventDestroy(fork);
  for (auto &c : pools) {
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
  cudaFree(d_init_list);
  cudaFree(d_slot_best);
  cudaFree(d_slot_evals);
  cudaFree(d_slot_keys);
  cudaFree(d_slot_round);
  cudaFree(d_first_slot);
  cudaFree(d_n_slots);
  cudaFree(d_task_next);
  cudaFree(d_planes);
  cudaFree(d_err);
  cudaFree(d_seq);
  if (own_stream && s) cudaStreamDestroy(s);
}

namespace psaw {
namespace {

constexpr int kTableFactor = 15;  // visited-table slots per pivot x 10

// working set a request needs while admitted: its walks' visited tables as if
// all ran at once plus its round slots and chunk keys
size_t request_cost(const labs_problem &p, int rounds_per_launch) {
  const int D = (p.L + 1) / 2;
  const size_t table = (size_t)visited_table_cap(p.walk_len, kTableFactor) * key_words64(D) * 8;
  const size_t chunks = (size_t)(p.walks + 31) / 32;
  return (size_t)p.walks * table + (size_t)rounds_per_launch * (16 + chunks * kKeyWords * 4) + 256;
}

}  // namespace
}  // namespace psaw

// One scheduling step over the admitted requests: plan, launch, finalize, harvest.
labs_status labs_server::step(std::vector<int> &active) {
  // plan rounds per request and tasks per class
  const int rpl = cfg.rounds_per_launch;
  std::vector<uint32_t> first(cfg.max_active, 0), cnt(cfg.max_active, 0), slot_round;
  uint32_t nslots = 0;
  std::vector<std::vector<std::pair<double, BatchTask>>> tk(pools.size());
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int sl : active) {
      Request &r = *reqs[slot_ticket[sl]];
      const uint64_t fr = (uint64_t)r.p.walks * r.p.walk_len * (uint64_t)((r.p.L + 1) / 2);
      const uint64_t rem = r.p.step_budget > r.evals ? r.p.step_budget - r.evals : 0;
      uint64_t k = rem == 0 ? 1 : (rem + fr - 1) / fr;
      k = std::max<uint64_t>(1, std::min<uint64_t>(k, (uint64_t)rpl));
      first[sl] = nslots;
      cnt[sl] = (uint32_t)k;
      const uint32_t chunks = (uint32_t)((r.p.walks + 31) / 32);
      const double cost = (double)r.p.walk_len * ((r.p.L + 1) / 2) * r.W;
      for (uint32_t j = 0; j < k; ++j) {
        slot_round.push_back((uint32_t)(r.next_round + (int32_t)j));
        for (uint32_t ch = 0; ch < chunks; ++ch)
          tk[r.W - 1].push_back({cost, BatchTask{(uint32_t)sl, (uint32_t)(r.next_round + (int32_t)j), ch, nslots + j}});
      }
      nslots += (uint32_t)k;
    }
  }
  for (size_t ci = 0; ci < pools.size(); ++ci) {
    ClassPool &c = pools[ci];
    auto &v = tk[ci];
    using Costed = std::pair<double, BatchTask>;
    std::stable_sort(v.begin(), v.end(), [](const Costed &x, const Costed &y) {
      return x.first > y.first;
    });
    c.n_tasks = (uint32_t)v.size();
    if (v.empty()) continue;
    if (v.size() > c.tasks_cap) {
      cudaFree(c.tasks);
      c.tasks_cap = std::max(v.size(), 2 * c.tasks_cap);
      if (dalloc(&c.tasks, c.tasks_cap) != cudaSuccess) return LABS_ENOMEM;
    }
    std::vector<BatchTask> flat(v.size());
    for (size_t j = 0; j < v.size(); ++j) flat[j] = v[j].second;
    if (cudaMemcpyAsync(c.tasks, flat.data(), sizeof(BatchTask) * flat.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return LABS_ECUDA;
  }
  if (cudaMemcpyAsync(d_slot_round, slot_round.data(), sizeof(uint32_t) * slot_round.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(d_first_slot, first.data(), sizeof(uint32_t) * first.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(d_n_slots, cnt.data(), sizeof(uint32_t) * cnt.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(d_slot_best, 0xFF, sizeof(unsigned long long) * nslots, s) != cudaSuccess ||
      cudaMemsetAsync(d_slot_evals, 0, sizeof(unsigned long long) * nslots, s) != cudaSuccess ||
      cudaMemsetAsync(d_task_next, 0, sizeof(unsigned int) * pools.size(), s) != cudaSuccess)
    return LABS_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  if (cudaEventRecord(fork, s) != cudaSuccess) return LABS_ECUDA;
  for (size_t ci = 0; ci < pools.size(); ++ci) {
    ClassPool &c = pools[ci];
    if (!c.n_tasks) continue;
    if (cudaStreamWaitEvent(cs[ci], fork, 0) != cudaSuccess) return LABS_ECUDA;
    BatchKernelParams k{};
    k.probs = d_probs;
    k.tasks = c.tasks;
    k.n_tasks = c.n_tasks;
    k.task_next = d_task_next + ci;
    k.pool = c.pool;
    k.pool_words = c.words;
    k.slot_best = d_slot_best;
    k.slot_evals = d_slot_evals;
    k.slot_keys = d_slot_keys;
    k.max_chunks = max_chunks;
    k.done = d_done;
    k.mul_one = 1u;
    k.mul_two = 2u;
    k.mul_four = 4u;
    k.mul_h31 = 0x80000000u;
    k.mul_h30 = 0x40000000u;
    k.plane_steps = d_planes;
    k.err = d_err;
    if (launch_batch(c.W, cfg.block_threads, k, cs[ci], nullptr) != cudaSuccess) return LABS_ECUDA;
    if (cudaEventRecord(cs_done[ci], cs[ci]) != cudaSuccess || cudaStreamWaitEvent(s, cs_done[ci], 0) != cudaSuccess)
      return LABS_ECUDA;
    ++walk_launches;
    ++launches;
  }
  BatchFinalizeParams f{};
  f.n_problems = cfg.max_active;
  f.first_slot = d_first_slot;
  f.n_slots = d_n_slots;
  f.slot_round = d_slot_round;
  f.slot_best = d_slot_best;
  f.slot_evals = d_slot_evals;
  f.slot_keys = d_slot_keys;
  f.max_chunks = max_chunks;
  f.budget = d_budget;
  f.target = d_target;
  f.done = d_done;
  f.bestE = d_bestE;
  f.key = d_key;
  f.best_round = d_best_round;
  f.best_walk = d_best_walk;
  f.evals = d_evals;
  f.rounds = d_rounds;
  if (launch_batch_finalize(f, s) != cudaSuccess) return LABS_ECUDA;
  ++launches;
  cudaEventRecord(e1, s);
  // harvest
  const int n = cfg.max_active;
  std::vector<int32_t> done(n), rounds(n);
  std::vector<int64_t> bestE(n);
  std::vector<unsigned long long> evals(n);
  int32_t err = 0;
  std::vector<unsigned long long> run_evals(nslots);
  if (cudaMemcpyAsync(run_evals.data(), d_slot_evals, sizeof(unsigned long long) * nslots, cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(done.data(), d_done, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(rounds.data(), d_rounds, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(bestE.data(), d_bestE, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(evals.data(), d_evals, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(&err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LABS_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  busy_ms += ms;
  if (err) return (err & kErrOverflow) ? LABS_EOVERFLOW : LABS_ECHECK;
  std::vector<int> finished_slots;
  for (int sl : active)
    if (done[sl]) finished_slots.push_back(sl);
  // sequences of the finished requests
  std::vector<std::vector<int8_t>> seqs(finished_slots.size());
  for (size_t i = 0; i < finished_slots.size(); ++i) {
    const int sl = finished_slots[i];
    int L;
    {
      std::lock_guard<std::mutex> lock(mu);
      L = reqs[slot_ticket[sl]]->p.L;
    }
    seqs[i].resize(L);
    if (launch_expand(1, L, d_key + (size_t)sl * kKeyWords, kKeyWords, d_seq, s) != cudaSuccess ||
        cudaMemcpyAsync(seqs[i].data(), d_seq, (size_t)L, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return LABS_ECUDA;
    ++launches;
  }
  const uint64_t t = now_ns();
  std::lock_guard<std::mutex> lock(mu);
  for (unsigned long long x : run_evals) evals_run += x;
  for (int sl : active) {
    Request &r = *reqs[slot_ticket[sl]];
    evals_done += evals[sl] - r.evals;
    r.evals = evals[sl];
    r.rounds = rounds[sl];
    r.next_round = rounds[sl];
    r.bestE = bestE[sl];
  }
  for (size_t i = 0; i < finished_slots.size(); ++i) {
    const int sl = finished_slots[i];
    Request &r = *reqs[slot_ticket[sl]];
    r.seq = std::move(seqs[i]);
    r.t_done = t;
    r.status = LABS_OK;
    r.slot = -1;
    mem_used -= r.mem_cost;
    slot_ticket[sl] = 0;
    ++n_completed;
  }
  if (!finished_slots.empty()) finished.notify_all();
  return LABS_OK;
}

void labs_server::loop() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<int> active, admitted;
    std::vector<BatchProblem> adm_probs;
    std::vector<uint64_t> adm_budget;
    std::vector<int64_t> adm_target;
    {
      std::unique_lock<std::mutex> lock(mu);
      for (;;) {
        if (stopping || failed != LABS_OK) break;
        // admit in arrival order while a slot is free and the working set fits
        while (!pending.empty()) {
          Request &r = *reqs[pending.front()];
          if (mem_used + r.mem_cost > cfg.mem_bytes) break;
          auto it = std::find(slot_ticket.begin(), slot_ticket.end(), 0ull);
          if (it == slot_ticket.end()) break;
          const int sl = (int)(it - slot_ticket.begin());
          *it = r.ticket;
          r.slot = sl;
          r.t_admit = now_ns();
          mem_used += r.mem_cost;
          pending.pop_front();
          admitted.push_back(sl);
          BatchProblem bp{};
          bp.L = r.p.L;
          bp.W = r.W;
          bp.walk_len = r.p.walk_len;
          bp.walks = r.p.walks;
          bp.cap = visited_table_cap(r.p.walk_len, kTableFactor);
          bp.kw64 = key_words64((r.p.L + 1) / 2);
          bp.seed = r.p.seed;
          adm_probs.push_back(bp);
          adm_budget.push_back(r.p.step_budget);
          adm_target.push_back(r.p.target_E);
        }
        for (int sl = 0; sl < cfg.max_active; ++sl)
          if (slot_ticket[sl]) active.push_back(sl);
        if (!active.empty()) break;
        wake.wait_for(lock, std::chrono::milliseconds(20));
      }
      if (stopping || failed != LABS_OK) {
        // shutdown: run nothing more; everything still queued or admitted ends with a status
        labs_status why = failed != LABS_OK ? failed : LABS_ESHUTDOWN;
        for (auto &kv : reqs)
          if (kv.second->status == LABS_PENDING) {
            kv.second->status = why;
            kv.second->t_done = now_ns();
          }
        pending.clear();
        std::fill(slot_ticket.begin(), slot_ticket.end(), 0ull);
        mem_used = 0;
        finished.notify_all();
        break;
      }
    }
    labs_status st = LABS_OK;
    if (!admitted.empty()) {
      // write the new requests into their slots and reset the slots' state
      for (size_t i = 0; i < admitted.size() && st == LABS_OK; ++i) {
        const int sl = admitted[i];
        if (cudaMemcpyAsync(d_probs + sl, &adm_probs[i], sizeof(BatchProblem), cudaMemcpyHostToDevice, s) ||
            cudaMemcpyAsync(d_budget + sl, &adm_budget[i], sizeof(uint64_t), cudaMemcpyHostToDevice, s) ||
            cudaMemcpyAsync(d_target + sl, &adm_target[i], sizeof(int64_t), cudaMemcpyHostToDevice, s))
          st = LABS_ECUDA;
      }
      if (st == LABS_OK &&
          (cudaMemcpyAsync(d_init_list, admitted.data(), sizeof(int32_t) * admitted.size(), cudaMemcpyHostToDevice,
                           s) != cudaSuccess ||
           launch_init_slots(d_init_list, (int)admitted.size(), d_bestE, d_evals, d_done, d_rounds, d_best_round,
                             d_best_walk, d_key, s) != cudaSuccess ||
           cudaStreamSynchronize(s) != cudaSuccess))
        st = LABS_ECUDA;
      ++launches;
    }
    if (st == LABS_OK) st = step(active);
    if (st != LABS_OK) {
      std::lock_guard<std::mutex> lock(mu);
      failed = st;
      for (auto &kv : reqs)
        if (kv.second->status == LABS_PENDING) {
          kv.second->status = st;
          kv.second->t_done = now_ns();
        }
      pending.clear();
      std::fill(slot_ticket.begin(), slot_ticket.end(), 0ull);
      mem_used = 0;
      finished.notify_all();
      break;
    }
  }
}

extern "C" void labs_serve_cfg_init(labs_serve_cfg *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->mem_bytes = (size_t)8 << 30;
  c->max_active = 64;
  c->max_L = 301;
  c->max_walks = 2048;
  c->max_walk_len = 0;
  c->rounds_per_launch = 8;  // measured: 8 beat 1, 2, 4 and 16 on throughput and median latency
  c->block_threads = 128;
}

extern "C" labs_status labs_serve_create(const labs_serve_cfg *cfg_in, labs_server **out) {
  if (!out) return LABS_EINVAL;
  *out = nullptr;
  labs_serve_cfg cfg;
  labs_serve_cfg_init(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.max_L == 0) cfg.max_L = 301;
  if (cfg.max_active <= 0 || cfg.max_active > 4096 || cfg.max_L < LABS_L_MIN || cfg.max_L > LABS_L_MAX ||
      !(cfg.max_L & 1) || cfg.max_walks <= 0 || cfg.max_walks > (1 << 20) || cfg.max_walk_len < 0 ||
      cfg.rounds_per_launch <= 0 || cfg.rounds_per_launch > 64 || cfg.block_threads < 32 ||
      cfg.block_threads > 256 || cfg.block_threads % 32 || cfg.mem_bytes == 0)
    return LABS_EINVAL;
  if (cfg.max_walk_len == 0) cfg.max_walk_len = 8 * ((cfg.max_L + 1) / 2);
  labs_server *sv = new (std::nothrow) labs_server();
  if (!sv) return LABS_ENOMEM;
  sv->cfg = cfg;
  sv->t_created = now_ns();
  auto fail = [&](labs_status e) {
    delete sv;
    return e;
  };
  if (cudaGetDevice(&sv->device) != cudaSuccess) return fail(LABS_ECUDA);
  if (cfg.stream) {
    sv->s = (cudaStream_t)cfg.stream;
  } else {
    if (cudaStreamCreateWithFlags(&sv->s, cudaStreamNonBlocking) != cudaSuccess) return fail(LABS_ECUDA);
    sv->own_stream = true;
  }
  const int n = cfg.max_active;
  sv->max_chunks = (uint32_t)((cfg.max_walks + 31) / 32);
  sv->max_slots = (uint32_t)n * (uint32_t)cfg.rounds_per_launch;
  sv->slot_ticket.assign(n, 0);
  if (dalloc(&sv->d_probs, n) || dalloc(&sv->d_budget, n) || dalloc(&sv->d_target, n) || dalloc(&sv->d_done, n) ||
      dalloc(&sv->d_best_round, n) || dalloc(&sv->d_best_walk, n) || dalloc(&sv->d_rounds, n) ||
      dalloc(&sv->d_bestE, n) || dalloc(&sv->d_key, (size_t)n * kKeyWords) || dalloc(&sv->d_evals, n) ||
      dalloc(&sv->d_init_list, n) || dalloc(&sv->d_slot_best, sv->max_slots) ||
      dalloc(&sv->d_slot_evals, sv->max_slots) ||
      dalloc(&sv->d_slot_keys, (size_t)sv->max_slots * sv->max_chunks * kKeyWords) ||
      dalloc(&sv->d_slot_round, sv->max_slots) || dalloc(&sv->d_first_slot, n) || dalloc(&sv->d_n_slots, n) ||
      dalloc(&sv->d_planes, 1) || dalloc(&sv->d_err, 1) || dalloc(&sv->d_seq, LABS_L_MAX + 1))
    return fail(LABS_ENOMEM);
  if (cudaMemset(sv->d_done, 0xFF, sizeof(int32_t) * n) != cudaSuccess ||  // free slots count as finished
      cudaMemset(sv->d_err, 0, sizeof(int32_t)) != cudaSuccess || cudaMemset(sv->d_planes, 0, 8) != cudaSuccess)
    return fail(LABS_ECUDA);
  // one visited-table pool per lag-word class up to max_L, sized for the
  // largest L and walk length that class accepts
  const int Wmax = lag_words(cfg.max_L);
  if (dalloc(&sv->d_task_next, Wmax)) return fail(LABS_ENOMEM);
  for (int W = 1; W <= Wmax; ++W) {
    ClassPool c;
    c.W = W;
    const int Lmax = std::min(cfg.max_L, 64 * W + 1);
    c.words = (size_t)visited_table_cap(cfg.max_walk_len, kTableFactor) * key_words64((Lmax + 1) / 2);
    c.words = (c.words + 1) / 2 * 2;
    c.resident = batch_resident_lanes(W, cfg.block_threads);
    if (c.resident <= 0) return fail(LABS_ECUDA);
    sv->pools.push_back(c);
    if (dalloc(&sv->pools.back().pool, (size_t)c.resident * c.words)) return fail(LABS_ENOMEM);
    cudaStream_t x;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return fail(LABS_ECUDA);
    sv->cs.push_back(x);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(LABS_ECUDA);
    sv->cs_done.push_back(e);
  }
  if (cudaEventCreateWithFlags(&sv->fork, cudaEventDisableTiming) != cudaSuccess) return fail(LABS_ECUDA);
  try {
    sv->th = std::thread([sv]() { sv->loop(); });
  } catch (...) {
    return fail(LABS_ENOMEM);
  }
  *out = sv;
  return LABS_OK;
}

extern "C" labs_status labs_serve_submit(labs_server *sv, const labs_problem *req, uint64_t *ticket) {
  if (!sv || !req || !ticket) return LABS_EINVAL;
  const labs_problem &p = *req;
  if (p.L < LABS_L_MIN || p.L > LABS_L_MAX || !(p.L & 1) || p.walks < 1 || p.walk_len < 1 || p.step_budget < 1)
    return LABS_EINVAL;
  // requests that can never be admitted
  if (p.L > sv->cfg.max_L || p.walks > sv->cfg.max_walks || p.walk_len > sv->cfg.max_walk_len ||
      request_cost(p, sv->cfg.rounds_per_launch) > sv->cfg.mem_bytes)
    return LABS_ENOMEM;
  auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
  if (!r) return LABS_ENOMEM;
  r->p = p;
  r->W = lag_words(p.L);
  r->mem_cost = request_cost(p, sv->cfg.rounds_per_launch);
  r->t_submit = now_ns();
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stopping) return LABS_ESHUTDOWN;
  if (sv->failed != LABS_OK) return sv->failed;
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->pending.push_back(r->ticket);
  sv->reqs[r->ticket] = std::move(r);
  ++sv->n_submitted;
  sv->wake.notify_one();
  return LABS_OK;
}

static void fill_result(const Request &r, labs_result *out, int8_t *best_seq) {
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->status = r.status;
    out->L = r.p.L;
    out->best_E = r.bestE;
    out->F = r.bestE > 0 ? (double)r.p.L * r.p.L / (2.0 * (double)r.bestE) : 0.0;
    out->evals = r.evals;
    out->rounds = r.rounds;
    out->reached_target = (r.p.target_E >= 0 && r.bestE >= 0 && r.bestE <= r.p.target_E) ? 1 : 0;
    out->t_submit_ns = r.t_submit;
    out->t_admit_ns = r.t_admit;
    out->t_done_ns = r.t_done;
    out->p_optimal = labs_model_p_optimal(r.p.L, labs_model_nses_of_evals(r.p.L, r.evals));
  }
  if (best_seq && r.status == LABS_OK) std::memcpy(best_seq, r.seq.data(), r.seq.size());
}

extern "C" labs_status labs_serve_poll(labs_server *sv, uint64_t ticket, labs_result *out, int8_t *best_seq) {
  if (!sv) return LABS_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return LABS_ENOTFOUND;
  Request &r = *it->second;
  if (r.status == LABS_PENDING) return LABS_PENDING;
  fill_result(r, out, best_seq);
  const labs_status st = r.status;
  sv->reqs.erase(it);
  return st;
}

extern "C" labs_status labs_serve_wait(labs_server *sv, uint64_t ticket, int64_t timeout_ms, labs_result *out,
                                       int8_t *best_seq) {
  if (!sv || timeout_ms < 0) return LABS_EINVAL;
  std::unique_lock<std::mutex> lock(sv->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return LABS_ENOTFOUND;
    Request &r = *it->second;
    if (r.status != LABS_PENDING) {
      fill_result(r, out, best_seq);
      const labs_status st = r.status;
      sv->reqs.erase(it);
      return st;
    }
    if (sv->finished.wait_until(lock, deadline) == std::cv_status::timeout) {
      auto it2 = sv->reqs.find(ticket);
      if (it2 != sv->reqs.end() && it2->second->status == LABS_PENDING) return LABS_ETIMEOUT;
    }
  }
}

extern "C" labs_status labs_serve_get_stats(labs_server *sv, labs_serve_stats *out) {
  if (!sv || !out) return LABS_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = sv->n_submitted;
  out->completed = sv->n_completed;
  out->pending = sv->pending.size();
  int act = 0;
  for (auto t : sv->slot_ticket) act += t != 0;
  out->active = (uint64_t)act;
  out->evals = sv->evals_done;
  out->evals_run = sv->evals_run;
  out->launches = sv->launches;
  out->walk_launches = sv->walk_launches;
  out->busy_ms = sv->busy_ms;
  out->mem_used = sv->mem_used;
  out->status = sv->failed;
  return LABS_OK;
}

extern "C" labs_status labs_serve_destroy(labs_server *sv) {
  if (!sv) return LABS_EINVAL;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stopping = true;
    sv->wake.notify_all();
  }
  if (sv->th.joinable()) sv->th.join();
  cudaStreamSynchronize(sv->s);
  delete sv;
  return LABS_OK;
}
