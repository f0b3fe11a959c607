// Serving loop with continuous batching (labs_serve_* in include/labs.h).
//
// Requests (one problem each) arrive at any time.  A scheduler thread admits
// them in arrival order into device slots while a slot is free and a launch
// over every admitted request still fits its half of the server's arena, and
// keeps two launches of the persistent batch kernels in flight: while one
// runs, the next is already queued on its own streams, so its tasks start on
// the SMs the first one's tail frees and the device never drains between
// launches.  Each launch gives every admitted request its next few rounds.
// The kernels finalize each request round by round as its rounds complete
// (Algorithm 1's best update and stop rule) and skip the rounds issued past a
// request's stop.  After a launch completes, the scheduler reads a snapshot of
// every admitted request, hands finished ones back, admits new ones and queues
// the next launch.  A request's result depends only on its own (L, seed,
// walks, walk_len, budget, target): the same alone and in any mix.
//
// Device memory: a fixed block of per-slot state and round records (sized by
// max_active, rounds_per_launch and max_walks), and an arena of mem_bytes
// whose two halves hold the task lists and visited-table pools of the two
// launches in flight.  Admission keeps every launch inside its half, so the
// bytes in use are bounded by mem_bytes whatever arrives.
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

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr int kSeqStride = 512;  // bytes per slot of the expanded best sequences (>= LABS_L_MAX)
constexpr int kDepth = 2;        // launches in flight
constexpr int kRingFactor = 6;   // round records per slot = kRingFactor x rounds_per_launch
// Warp mode keeps a key slot per walk in every round record: it is offered
// while max_walks is at most this.
constexpr int kWarpModeMaxWalks = 4096;

struct Request {
  uint64_t ticket = 0;
  labs_problem p{};
  int W = 0;
  uint64_t t_submit = 0, t_admit = 0, t_done = 0;
  labs_status status = LABS_PENDING;
  int slot = -1;
  // the host's view, from the latest snapshot that listed the request
  int64_t bestE = -1;
  uint64_t evals = 0, planes = 0;
  int32_t rounds = 0;          // rounds finalized
  uint32_t issued = 0;         // next round to issue
  uint64_t first_launch = 0;   // the first launch that lists it
  std::vector<int8_t> seq;
};

// What one launch runs for one request: its rounds (k) and the sizes that
// decide the launch's device memory.
struct Share {
  int slot, W, L, walk_len, walks;
  uint32_t k, chunks;
  size_t table_words;  // 64-bit words of one walk's visited table
};

Share share_of(int slot, const labs_problem &p, uint32_t k) {
  Share s;
  s.slot = slot;
  s.W = lag_words(p.L);
  s.L = p.L;
  s.walk_len = p.walk_len;
  s.walks = p.walks;
  s.k = k;
  s.chunks = (uint32_t)((p.walks + 31) / 32);
  s.table_words = (size_t)visited_table_cap(p.walk_len) * (size_t)key_words64((p.L + 1) / 2);
  s.table_words = (s.table_words + 1) / 2 * 2;  // whole 16-byte units (the warp clears in uint4)
  return s;
}

// Evaluations per second of one mode of a class as a function of the warps
// its tasks occupy: measured at kLevels occupancies (when the server is
// created) and interpolated linearly between (0, 0) and those points, flat past
// the last.  Throughput is not proportional to the warps busy: it saturates as
// the SMs fill, so the choice between modes needs the curve, not one rate.
constexpr int kLevels = 3;
struct Curve {
  double warps[kLevels] = {0, 0, 0}, evals_per_s[kLevels] = {0, 0, 0};
  double at(double n) const {
    double x0 = 0, y0 = 0;
    for (int i = 0; i < kLevels; ++i) {
      if (n <= warps[i]) return warps[i] > x0 ? y0 + (evals_per_s[i] - y0) * (n - x0) / (warps[i] - x0) : y0;
      x0 = warps[i];
      y0 = evals_per_s[i];
    }
    return y0;
  }
};

// The kernel variants a launch can run a class with (batch.cuh): one walk per
// lane, the same with the scan's flip loop unrolled twice, one walk per warp.
constexpr int kModes = 3;
constexpr int kModeVariant[kModes] = {kBatchLane, kBatchLaneUnroll2, kBatchWarp};
inline bool mode_is_warp(int m) { return kModeVariant[m] == kBatchWarp; }

// What the scheduler knows of each lag-word class: per mode, the tables (lanes,
// or warps in warp mode) its kernel keeps resident, whether it is offered, and
// its throughput curve.
struct ClassInfo {
  int resident[kModes] = {0, 0, 0};
  bool offered[kModes] = {false, false, false};
  Curve curve[kModes];
  int forced = 0;  // 1: always one walk per lane, 2: always one walk per warp
};

// The mode for a class in one launch: the one whose curve is highest at the
// warps the launch's tasks occupy (one walk per lane fills a warp per 32
// walks, one walk per warp a warp per walk).  Another mode replaces the plain
// lane mode only when its curve is kModeMargin higher: the curves come from
// short samples, and a choice within their noise would trade away a sure
// result for a guess.
constexpr double kModeMargin = 1.05;
int choose_mode(const ClassInfo &ci, uint64_t chunk_tasks, uint64_t walk_tasks) {
  if (ci.forced == 2) return 2;
  int best = 0;
  double best_rate = -1.0;
  for (int m = 0; m < kModes; ++m) {
    if (!ci.offered[m] || (ci.forced == 1 && mode_is_warp(m))) continue;
    const uint64_t warps = mode_is_warp(m) ? std::min<uint64_t>(walk_tasks, (uint64_t)ci.resident[m])
                                           : std::min<uint64_t>(chunk_tasks, (uint64_t)ci.resident[m] / 32);
    const double rate = ci.curve[m].at((double)warps) * (m == 0 ? kModeMargin : 1.0);
    if (rate > best_rate) {
      best_rate = rate;
      best = m;
    }
  }
  return best;
}

// Layout of one launch inside its half of the arena (byte offsets; sizes
// only when computed for admission): the lists uploaded from the host (the
// listed problems, the records to issue, the task list of each class), then
// one visited-table pool per class with a table for each lane (or warp, in
// warp mode) that can run one of its tasks at once.
struct Carve {
  size_t problems = 0, issue = 0, recs = 0;
  std::vector<size_t> tasks;  // per class
  size_t upload_bytes = 0;
  std::vector<size_t> pool;        // per class
  std::vector<size_t> pool_words;  // per class, per lane
  std::vector<int> lanes;          // per class: lanes, or warps in warp mode, of the grid
  std::vector<uint32_t> n_tasks;   // per class
  std::vector<uint8_t> mode;       // per class: the kernel variant (kModeVariant)
  uint32_t n_problems = 0, n_issue = 0;
  size_t total = 0;
};

Carve carve_launch(const std::vector<Share> &sh, const std::vector<ClassInfo> &cls, int block) {
  const size_t nc = cls.size();
  Carve c;
  c.tasks.assign(nc, 0);
  c.pool.assign(nc, 0);
  c.pool_words.assign(nc, 0);
  c.lanes.assign(nc, 0);
  c.n_tasks.assign(nc, 0);
  c.mode.assign(nc, 0);
  c.n_problems = (uint32_t)sh.size();
  std::vector<uint64_t> chunk_tasks(nc, 0), walk_tasks(nc, 0);
  for (const Share &s : sh) {
    c.n_issue += s.k;
    chunk_tasks[s.W - 1] += (uint64_t)s.k * s.chunks;
    walk_tasks[s.W - 1] += (uint64_t)s.k * (uint64_t)s.walks;
    if (s.k) c.pool_words[s.W - 1] = std::max(c.pool_words[s.W - 1], s.table_words);
  }
  for (size_t w = 0; w < nc; ++w) {
    c.mode[w] = (uint8_t)choose_mode(cls[w], chunk_tasks[w], walk_tasks[w]);
    c.n_tasks[w] = (uint32_t)(mode_is_warp(c.mode[w]) ? walk_tasks[w] : chunk_tasks[w]);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  c.problems = take(sizeof(int32_t) * c.n_problems);
  c.issue = take(sizeof(RecordInit) * c.n_issue);
  c.recs = take(sizeof(uint32_t) * c.n_issue);
  for (size_t w = 0; w < nc; ++w) c.tasks[w] = take(sizeof(BatchTask) * c.n_tasks[w]);
  c.upload_bytes = off;
  for (size_t w = 0; w < nc; ++w) {
    if (!c.n_tasks[w]) continue;
    // a table per lane (32 per task) or per warp (one per task), whole CTAs, at most the resident ones
    const bool warp = mode_is_warp(c.mode[w]);
    const size_t per_block = warp ? (size_t)block / 32 : (size_t)block;
    const size_t units = warp ? (size_t)c.n_tasks[w] : (size_t)c.n_tasks[w] * 32;
    const size_t want = (units + per_block - 1) / per_block * per_block;
    c.lanes[w] = (int)std::min<size_t>(want, (size_t)cls[w].resident[c.mode[w]]);
    c.pool[w] = take(sizeof(uint64_t) * c.pool_words[w] * (size_t)c.lanes[w]);
  }
  c.total = off;
  return c;
}

// One of the launches in flight: its streams, events, arena half and snapshot.
struct Launch {
  uint64_t id = 0;
  bool in_flight = false;
  cudaStream_t s = nullptr;
  std::vector<cudaStream_t> cs;
  std::vector<cudaEvent_t> cs_done;
  cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr;
  char *arena = nullptr;
  unsigned int *task_next = nullptr;  // per class
  int32_t *init_list = nullptr;       // the slots this launch starts afresh
  int32_t *snap_err = nullptr;        // the error word, copied before the read-back
  char *d_snap = nullptr, *h_snap = nullptr;  // h_snap: pinned
  size_t snap_bytes = 0;
  Snapshot snap{};
  std::vector<int> slots;   // the slots it lists
  size_t carve_bytes = 0;
  int walk_kernels = 0;
};

}  // namespace
}  // namespace psaw

using namespace psaw;

struct labs_server {
  labs_serve_cfg cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable wake;       // scheduler: new request or shutdown
  std::condition_variable finished;   // waiters: a request finished
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<uint64_t> slot_ticket;     // 0 = free
  std::vector<uint64_t> slot_listed;     // the last launch that listed the slot
  std::vector<uint8_t> slot_draining;    // finished, but a launch in flight still lists it
  size_t mem_used = 0, mem_peak = 0, fixed_bytes = 0, half_bytes = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  labs_status failed = LABS_OK;
  std::thread th;
  // counters
  uint64_t n_submitted = 0, n_completed = 0, evals_done = 0, evals_run = 0;
  uint64_t launches = 0, walk_launches = 0;
  uint64_t mode_launches[kModes] = {0, 0, 0};  // class kernels launched in each mode
  double busy_ms = 0.0, busy_end_ms = 0.0;
  // device state
  void *fixed = nullptr;
  BatchProblem *d_probs = nullptr;
  ProblemState ps{};
  RoundRecords rec{};
  int32_t *d_err = nullptr;
  uint32_t ring = 0;
  char *arena = nullptr;
  std::vector<ClassInfo> cls;  // per class W - 1
  bool warp_allowed = false;
  Launch L[kDepth];
  cudaEvent_t t_ref = nullptr;
  uint64_t harvested = 0;  // id of the last launch harvested

  ~labs_server();
  void loop();
  void fail_all(labs_status why);
  size_t admitted_carve(const Request *extra);                      // caller holds mu
  labs_status enqueue(Launch &l, const std::vector<int> &admitted);  // caller does not hold mu
  labs_status harvest(Launch &l);
  labs_status tune_modes();
  uint32_t tune_record = 0;
};

labs_server::~labs_server() {
  for (auto &l : L) {
    for (auto x : l.cs) cudaStreamDestroy(x);
    for (auto e : l.cs_done) cudaEventDestroy(e);
    if (l.fork) cudaEventDestroy(l.fork);
    if (l.ev0) cudaEventDestroy(l.ev0);
    if (l.ev1) cudaEventDestroy(l.ev1);
    if (l.s) cudaStreamDestroy(l.s);
    cudaFree(l.d_snap);
    cudaFreeHost(l.h_snap);
  }
  if (t_ref) cudaEventDestroy(t_ref);
  cudaFree(fixed);
  cudaFree(arena);
}

// Arena bytes of one launch over every admitted request (and `extra`), each
// running rounds_per_launch rounds (the most a launch gives a request).
size_t labs_server::admitted_carve(const Request *extra) {
  std::vector<Share> sh;
  for (int sl = 0; sl < cfg.max_active; ++sl)
    if (slot_ticket[sl] && !slot_draining[sl])
      sh.push_back(share_of(sl, reqs[slot_ticket[sl]]->p, (uint32_t)cfg.rounds_per_launch));
  if (extra) sh.push_back(share_of(-1, extra->p, (uint32_t)cfg.rounds_per_launch));
  return carve_launch(sh, cls, cfg.block_threads).total;
}

// Rounds the next launch gives a request: what its budget still needs beyond
// the rounds in flight, at most `most`, and never so far ahead of the
// finalized rounds that the ring would reuse a record still in use.
static uint32_t rounds_to_issue(const Request &r, int64_t most, uint32_t ring) {
  const uint64_t fr = (uint64_t)r.p.walks * (uint64_t)r.p.walk_len * (uint64_t)((r.p.L + 1) / 2);
  const uint64_t rem = r.p.step_budget > r.evals ? r.p.step_budget - r.evals : 0;
  const int64_t need = (int64_t)std::max<uint64_t>(1, (rem + fr - 1) / fr);
  const int64_t in_flight = (int64_t)r.issued - (int64_t)r.rounds;
  const int64_t room = (int64_t)r.rounds + (int64_t)ring - (int64_t)r.issued;
  const int64_t k = std::min<int64_t>({need - in_flight, room, most});
  return k > 0 ? (uint32_t)k : 0u;
}

// Rounds per request of one launch.  Each gets rounds_per_launch (or what it
// still needs); when those leave SMs idle (few requests, or the last ones of
// a burst), requests get further rounds, one at a time in turn, until the
// launch's warps reach what the device keeps resident of its widest-fitting
// class or no request can take more.  The further rounds mostly run on lanes
// that would otherwise idle (the saturated throughput measured the same with
// and without them), and a request that needs them finishes in fewer
// launches.  Targets still stop every request at the same round.
static std::vector<uint32_t> plan_rounds(const std::vector<const Request *> &rs, int rounds_per_launch,
                                         uint32_t ring, const std::vector<ClassInfo> &cls) {
  std::vector<uint32_t> k(rs.size());
  uint64_t warps = 0, fill = 0;
  for (size_t i = 0; i < rs.size(); ++i) {
    k[i] = rounds_to_issue(*rs[i], rounds_per_launch, ring);
    const uint64_t chunks = (uint64_t)((rs[i]->p.walks + 31) / 32);
    warps += k[i] * chunks;
    fill = std::max<uint64_t>(fill, (uint64_t)cls[rs[i]->W - 1].resident[0] / 32);
  }
  for (bool grew = true; grew && warps < fill;) {
    grew = false;
    for (size_t i = 0; i < rs.size() && warps < fill; ++i) {
      if (k[i] == 0 || rounds_to_issue(*rs[i], (int64_t)k[i] + 1, ring) <= k[i]) continue;
      ++k[i];
      warps += (uint64_t)((rs[i]->p.walks + 31) / 32);
      grew = true;
    }
  }
  return k;
}

// Plan and queue one launch on l's streams: the new requests' slot state, the
// records of the rounds issued, the class kernels, the finalization of what
// they left, and the snapshot of every listed slot with its read-back.
labs_status labs_server::enqueue(Launch &l, const std::vector<int> &admitted) {
  const int rpl = cfg.rounds_per_launch;
  std::vector<Share> sh;
  std::vector<int64_t> target(cfg.max_active, -1);
  std::vector<uint32_t> first_round(cfg.max_active, 0);
  std::vector<BatchProblem> adm_probs;
  std::vector<uint64_t> adm_budget;
  std::vector<int64_t> adm_target;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int sl : admitted) {
      const Request &r = *reqs[slot_ticket[sl]];
      BatchProblem bp{};
      bp.L = r.p.L;
      bp.W = r.W;
      bp.walk_len = r.p.walk_len;
      bp.walks = r.p.walks;
      bp.cap = visited_table_cap(r.p.walk_len);
      bp.kw64 = key_words64((r.p.L + 1) / 2);
      bp.seed = r.p.seed;
      adm_probs.push_back(bp);
      adm_budget.push_back(r.p.step_budget);
      adm_target.push_back(r.p.target_E);
    }
    l.slots.clear();
    std::vector<const Request *> listed;
    for (int sl = 0; sl < cfg.max_active; ++sl)
      if (slot_ticket[sl] && !slot_draining[sl]) listed.push_back(reqs[slot_ticket[sl]].get());
    std::vector<uint32_t> ks = plan_rounds(listed, rpl, ring, cls);
    {  // the further rounds only while the launch stays inside its half of the arena
      std::vector<Share> trial;
      for (size_t i = 0; i < listed.size(); ++i) trial.push_back(share_of(listed[i]->slot, listed[i]->p, ks[i]));
      if (carve_launch(trial, cls, cfg.block_threads).total > half_bytes)
        for (size_t i = 0; i < listed.size(); ++i) ks[i] = rounds_to_issue(*listed[i], rpl, ring);
    }
    size_t li = 0;
    for (int sl = 0; sl < cfg.max_active; ++sl) {
      if (!slot_ticket[sl] || slot_draining[sl]) continue;
      Request &r = *reqs[slot_ticket[sl]];
      const uint32_t k = ks[li++];
      sh.push_back(share_of(sl, r.p, k));
      target[sl] = r.p.target_E;
      first_round[sl] = r.issued;
      r.issued += k;
      if (!r.first_launch) r.first_launch = l.id;
      slot_listed[sl] = l.id;
      l.slots.push_back(sl);
    }
  }
  const Carve cv = carve_launch(sh, cls, cfg.block_threads);
  if (cv.total > half_bytes) return LABS_ENOMEM;  // admission keeps this from happening
  l.carve_bytes = cv.total;
  // the uploaded lists
  std::vector<char> up(cv.upload_bytes);
  int32_t *plist = reinterpret_cast<int32_t *>(up.data() + cv.problems);
  RecordInit *ilist = reinterpret_cast<RecordInit *>(up.data() + cv.issue);
  uint32_t *rlist = reinterpret_cast<uint32_t *>(up.data() + cv.recs);
  std::vector<std::vector<PlannedTask>> tk(cls.size());
  size_t ni = 0;
  for (size_t i = 0; i < sh.size(); ++i) {
    const Share &s = sh[i];
    plist[i] = s.slot;
    const double cost = batch_task_cost(s.L, s.walk_len);
    const bool layered = target[s.slot] >= 0;
    const bool warp = mode_is_warp(cv.mode[s.W - 1]);
    const uint32_t units = warp ? (uint32_t)s.walks : s.chunks;  // tasks per round: walks, or chunks of 32
    for (uint32_t j = 0; j < s.k; ++j) {
      const uint32_t round = first_round[s.slot] + j;
      const uint32_t recx = (uint32_t)s.slot * ring + round % ring;
      ilist[ni] = RecordInit{recx, round, units, warp ? 0u : 5u};
      rlist[ni] = recx;
      ++ni;
      for (uint32_t u = 0; u < units; ++u)
        tk[s.W - 1].push_back({layered ? j : 0u, cost, BatchTask{(uint32_t)s.slot, round, u, recx}});
    }
  }
  for (size_t ci = 0; ci < tk.size(); ++ci) {
    order_tasks(tk[ci]);
    BatchTask *dst = reinterpret_cast<BatchTask *>(up.data() + cv.tasks[ci]);
    for (size_t j = 0; j < tk[ci].size(); ++j) dst[j] = tk[ci][j].t;
  }
  cudaStream_t s = l.s;
  char *a = l.arena;
  const int32_t *d_plist = reinterpret_cast<const int32_t *>(a + cv.problems);
  // new requests: their problem, budget and target, then a fresh state
  for (size_t i = 0; i < admitted.size(); ++i) {
    const int sl = admitted[i];
    if (cudaMemcpyAsync(d_probs + sl, &adm_probs[i], sizeof(BatchProblem), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(const_cast<uint64_t *>(ps.budget) + sl, &adm_budget[i], sizeof(uint64_t),
                        cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(const_cast<int64_t *>(ps.target) + sl, &adm_target[i], sizeof(int64_t),
                        cudaMemcpyHostToDevice, s))
      return LABS_ECUDA;
  }
  if (cudaMemcpyAsync(a, up.data(), up.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) return LABS_ECUDA;
  if (!admitted.empty()) {
    if (cudaMemcpyAsync(l.init_list, admitted.data(), sizeof(int32_t) * admitted.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        launch_init_problems_state(l.init_list, (int)admitted.size(), rec, ps, s) != cudaSuccess)
      return LABS_ECUDA;
    ++launches;
  }
  if (cudaEventRecord(l.ev0, s) != cudaSuccess ||
      launch_issue_records(reinterpret_cast<const RecordInit *>(a + cv.issue), (int)cv.n_issue, rec, s) !=
          cudaSuccess ||
      cudaMemsetAsync(l.task_next, 0, sizeof(unsigned int) * cls.size(), s) != cudaSuccess ||
      cudaEventRecord(l.fork, s) != cudaSuccess)
    return LABS_ECUDA;
  ++launches;
  l.walk_kernels = 0;
  for (size_t ci = 0; ci < cls.size(); ++ci) {
    if (!cv.n_tasks[ci]) continue;
    if (cudaStreamWaitEvent(l.cs[ci], l.fork, 0) != cudaSuccess) return LABS_ECUDA;
    BatchKernelParams k{};
    k.probs = d_probs;
    k.tasks = reinterpret_cast<const BatchTask *>(a + cv.tasks[ci]);
    k.n_tasks = cv.n_tasks[ci];
    k.task_next = l.task_next + ci;
    k.pool = reinterpret_cast<uint64_t *>(a + cv.pool[ci]);
    k.pool_words = cv.pool_words[ci];
    k.rec = rec;
    k.ps = ps;
    k.mul_one = 1u;
    k.mul_two = 2u;
    k.mul_four = 4u;
    k.mul_h31 = 0x80000000u;
    k.mul_h30 = 0x40000000u;
    k.err = d_err;
    // the pool holds cv.lanes[ci] tables: never more blocks than that
    const int variant = kModeVariant[cv.mode[ci]];
    const cudaError_t e =
        variant == kBatchWarp
            ? launch_batch_warp((int)ci + 1, cfg.block_threads, k, l.cs[ci], cv.lanes[ci] / (cfg.block_threads / 32))
            : launch_batch((int)ci + 1, cfg.block_threads, k, l.cs[ci], nullptr, cv.lanes[ci] / cfg.block_threads,
                           variant == kBatchLaneUnroll2 ? 2 : 1);
    if (e != cudaSuccess) return LABS_ECUDA;
    ++mode_launches[cv.mode[ci]];
    if (cudaEventRecord(l.cs_done[ci], l.cs[ci]) != cudaSuccess ||
        cudaStreamWaitEvent(s, l.cs_done[ci], 0) != cudaSuccess)
      return LABS_ECUDA;
    ++l.walk_kernels;
  }
  walk_launches += (uint64_t)l.walk_kernels;
  launches += (uint64_t)l.walk_kernels;
  if (cudaMemsetAsync(l.snap.run_evals, 0, sizeof(unsigned long long), s) != cudaSuccess ||
      launch_batch_finalize(d_plist, (int)cv.n_problems, rec, ps, s) != cudaSuccess ||
      launch_snapshot(d_plist, (int)cv.n_problems, d_probs, ps, reinterpret_cast<const uint32_t *>(a + cv.recs),
                      (int)cv.n_issue, rec, l.snap, s) != cudaSuccess)
    return LABS_ECUDA;
  launches += 2;
  if (cudaMemcpyAsync(l.snap_err, d_err, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(l.h_snap, l.d_snap, l.snap_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaEventRecord(l.ev1, s) != cudaSuccess)
    return LABS_ECUDA;
  l.in_flight = true;
  return LABS_OK;
}

// Take in a completed launch's snapshot: every listed request's progress;
// finished requests get their results; slots no launch in flight lists any
// more become free.
labs_status labs_server::harvest(Launch &l) {
  if (cudaEventSynchronize(l.ev1) != cudaSuccess) return LABS_ECUDA;
  l.in_flight = false;
  float t0 = 0.f, t1 = 0.f;
  cudaEventElapsedTime(&t0, t_ref, l.ev0);
  cudaEventElapsedTime(&t1, t_ref, l.ev1);
  auto at = [&](const void *dev) { return l.h_snap + ((const char *)dev - l.d_snap); };
  const int32_t err = *reinterpret_cast<const int32_t *>(at(l.snap_err));
  if (err & kErrOverflow) return LABS_EOVERFLOW;
  if (err & kErrRecheck) return LABS_ECHECK;
  if (err) return LABS_ECUDA;
  const int32_t *done = reinterpret_cast<const int32_t *>(at(l.snap.done));
  const int32_t *rounds = reinterpret_cast<const int32_t *>(at(l.snap.rounds));
  const int64_t *bestE = reinterpret_cast<const int64_t *>(at(l.snap.bestE));
  const unsigned long long *evals = reinterpret_cast<const unsigned long long *>(at(l.snap.evals));
  const unsigned long long *planes = reinterpret_cast<const unsigned long long *>(at(l.snap.planes));
  const int8_t *seqs = reinterpret_cast<const int8_t *>(at(l.snap.seq));
  const unsigned long long run = *reinterpret_cast<const unsigned long long *>(at(l.snap.run_evals));
  const uint64_t t = now_ns();
  std::lock_guard<std::mutex> lock(mu);
  harvested = l.id;
  // device time: the union of the launches' intervals
  const double b0 = std::max<double>(t0, busy_end_ms);
  if (t1 > b0) busy_ms += t1 - b0;
  busy_end_ms = std::max<double>(busy_end_ms, t1);
  mem_peak = std::max(mem_peak, l.carve_bytes);
  evals_run += run;
  bool any = false;
  for (int sl : l.slots) {
    if (!slot_ticket[sl] || slot_draining[sl]) continue;
    Request &r = *reqs[slot_ticket[sl]];
    // launches overlap, so a snapshot can be older than one already taken in:
    // keep the view that has the most rounds finalized
    if (rounds[sl] < r.rounds || (rounds[sl] == r.rounds && !done[sl] && r.rounds > 0)) continue;
    {
      evals_done += evals[sl] - r.evals;
      r.evals = evals[sl];
      r.planes = planes[sl];
      r.rounds = rounds[sl];
      r.bestE = bestE[sl];
      if (done[sl]) {
        r.seq.assign(seqs + (size_t)sl * kSeqStride, seqs + (size_t)sl * kSeqStride + r.p.L);
        r.t_done = t;
        r.status = LABS_OK;
        ++n_completed;
        any = true;
        slot_draining[sl] = 1;
      }
    }
  }
  // a finished request's slot is free once no launch in flight lists it
  for (int sl = 0; sl < cfg.max_active; ++sl) {
    if (slot_ticket[sl] && slot_draining[sl] && slot_listed[sl] <= harvested) {
      slot_ticket[sl] = 0;
      slot_draining[sl] = 0;
    }
  }
  mem_used = admitted_carve(nullptr);
  if (any) finished.notify_all();
  return LABS_OK;
}

// Measure, for every class, the throughput curve of each kernel mode (one
// walk per lane, the same unrolled, one walk per warp): evaluations per
// second with 1/8, 1/2 and all of the warps each mode
// keeps resident busy (as far as half the arena holds their tables), on a
// sample problem (the class's largest L up to max_L, walks of 128 steps, a
// round no request uses).  Slot 0 holds the sample problem meanwhile; the
// sample's tasks count into one record that never completes.
labs_status labs_server::tune_modes() {
  Launch &l = L[0];
  cudaStream_t s = l.s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LABS_ECUDA;
  labs_status st = LABS_OK;
  for (size_t ci = 0; ci < cls.size() && st == LABS_OK; ++ci) {
    const int W = (int)ci + 1;
    const int L = std::min(cfg.max_L, 64 * W + 1);
    const int D = (L + 1) / 2;
    BatchProblem pr{};
    pr.L = L;
    pr.W = W;
    pr.walk_len = std::min(8 * D, 128);
    pr.walks = std::max({cls[ci].resident[0], cls[ci].resident[1], cls[ci].resident[2]});
    pr.cap = visited_table_cap(pr.walk_len);
    pr.kw64 = key_words64(D);
    pr.seed = 0x5EEDu;
    const size_t words = ((size_t)pr.cap * pr.kw64 + 1) / 2 * 2;
    const int32_t not_done = 0;
    if (cudaMemcpyAsync(d_probs, &pr, sizeof(pr), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ps.done, &not_done, sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = LABS_ECUDA;
      break;
    }
    for (int mode = 0; mode < kModes && st == LABS_OK; ++mode) {
      const bool warp = mode_is_warp(mode);
      cls[ci].offered[mode] = !warp || warp_allowed;
      if (!cls[ci].offered[mode]) continue;
      const int per_block = warp ? cfg.block_threads / 32 : cfg.block_threads;
      const int tables_per_warp = warp ? 1 : 32;
      const size_t resident_warps = (size_t)cls[ci].resident[mode] / tables_per_warp;
      Curve &cv = cls[ci].curve[mode];
      for (int lv = 0; lv < kLevels && st == LABS_OK; ++lv) {
        const size_t want = lv == 0 ? resident_warps / 8 : (lv == 1 ? resident_warps / 2 : resident_warps);
        size_t units = std::max<size_t>(1, want) * tables_per_warp;  // tables: lanes or warps
        const size_t task_bytes = align_up(sizeof(BatchTask) * units);
        const size_t fit = half_bytes > task_bytes ? (half_bytes - task_bytes) / (words * 8) : 0;
        units = std::min(units, fit);
        units = (units + per_block - 1) / per_block * per_block;
        if (units > fit) units -= per_block;
        const size_t n_tasks = units / tables_per_warp;
        if (n_tasks == 0) {
          if (lv == 0) cls[ci].offered[mode] = false;
          break;
        }
        std::vector<BatchTask> tk(n_tasks);
        for (size_t i = 0; i < n_tasks; ++i) tk[i] = BatchTask{0u, 1000000u, (uint32_t)i, tune_record};
        BatchKernelParams k{};
        k.probs = d_probs;
        k.tasks = reinterpret_cast<const BatchTask *>(l.arena);
        k.n_tasks = (uint32_t)n_tasks;
        k.task_next = l.task_next;
        k.pool = reinterpret_cast<uint64_t *>(l.arena + task_bytes);
        k.pool_words = words;
        k.rec = rec;
        k.ps = ps;
        k.mul_one = 1u;
        k.mul_two = 2u;
        k.mul_four = 4u;
        k.mul_h31 = 0x80000000u;
        k.mul_h30 = 0x40000000u;
        k.err = d_err;
        float ms = 0.f;
        unsigned long long evals = 0;
        if (cudaMemcpyAsync(l.arena, tk.data(), sizeof(BatchTask) * n_tasks, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
          st = LABS_ECUDA;
        for (int rep = 0; rep < 2 && st == LABS_OK; ++rep) {  // the first run warms up
          const cudaError_t e =
              (cudaMemsetAsync(l.task_next, 0, sizeof(unsigned int), s) != cudaSuccess ||
               cudaMemsetAsync(rec.left + tune_record, 0xFF, sizeof(uint32_t), s) != cudaSuccess ||
               cudaMemsetAsync(rec.evals + tune_record, 0, sizeof(unsigned long long), s) != cudaSuccess ||
               cudaEventRecord(e0, s) != cudaSuccess)
                  ? cudaErrorUnknown
                  : (warp ? launch_batch_warp(W, cfg.block_threads, k, s, (int)(units / per_block))
                          : launch_batch(W, cfg.block_threads, k, s, nullptr, (int)(units / per_block),
                                         kModeVariant[mode] == kBatchLaneUnroll2 ? 2 : 1));
          if (e != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
              cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = LABS_ECUDA;
        }
        if (st == LABS_OK &&
            cudaMemcpy(&evals, rec.evals + tune_record, sizeof(evals), cudaMemcpyDeviceToHost) != cudaSuccess)
          st = LABS_ECUDA;
        if (st != LABS_OK) break;
        cv.warps[lv] = (double)n_tasks;
        cv.evals_per_s[lv] = (double)evals / (std::max(ms, 1e-3f) / 1e3);
        for (int j = lv + 1; j < kLevels; ++j) {  // until measured, flat
          cv.warps[j] = cv.warps[lv];
          cv.evals_per_s[j] = cv.evals_per_s[lv];
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int32_t free_slot = 1;
  int32_t err = 0;
  if (st == LABS_OK &&
      (cudaMemcpyAsync(ps.done, &free_slot, sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(&err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    st = LABS_ECUDA;
  if (st == LABS_OK && err) st = (err & kErrOverflow) ? LABS_EOVERFLOW : LABS_ECUDA;
  return st;
}

void labs_server::fail_all(labs_status why) {
  std::lock_guard<std::mutex> lock(mu);
  if (failed == LABS_OK && why != LABS_ESHUTDOWN) failed = why;
  for (auto &kv : reqs)
    if (kv.second->status == LABS_PENDING) {
      kv.second->status = why;
      kv.second->t_done = now_ns();
    }
  pending.clear();
  std::fill(slot_ticket.begin(), slot_ticket.end(), 0ull);
  std::fill(slot_draining.begin(), slot_draining.end(), (uint8_t)0);
  mem_used = 0;
  finished.notify_all();
}

void labs_server::loop() {
  cudaSetDevice(device);
  std::deque<int> inflight;  // indices into L, oldest first
  uint64_t next_id = 1;
  labs_status st = LABS_OK;
  auto harvest_oldest = [&]() {
    st = harvest(L[inflight.front()]);
    inflight.pop_front();
  };
  for (;;) {
    bool stop;
    {
      std::lock_guard<std::mutex> lock(mu);
      stop = stopping;
    }
    if (stop || st != LABS_OK) break;
    // take in the launches that have completed, oldest first
    while (st == LABS_OK && !inflight.empty() && cudaEventQuery(L[inflight.front()].ev1) == cudaSuccess)
      harvest_oldest();
    if (st != LABS_OK) break;
    if ((int)inflight.size() == kDepth) {
      harvest_oldest();
      continue;
    }
    // admit in arrival order while a slot is free and a launch over all
    // admitted requests still fits its half of the arena
    std::vector<int> admitted;
    bool work = false;
    {
      std::lock_guard<std::mutex> lock(mu);
      while (!pending.empty()) {
        Request &r = *reqs[pending.front()];
        auto it = std::find(slot_ticket.begin(), slot_ticket.end(), 0ull);
        if (it == slot_ticket.end()) break;
        const size_t need = admitted_carve(&r);
        if (need > half_bytes) break;
        const int sl = (int)(it - slot_ticket.begin());
        *it = r.ticket;
        r.slot = sl;
        r.t_admit = now_ns();
        mem_used = need;
        pending.pop_front();
        admitted.push_back(sl);
      }
      for (int sl = 0; sl < cfg.max_active && !work; ++sl)
        if (slot_ticket[sl] && !slot_draining[sl] && rounds_to_issue(*reqs[slot_ticket[sl]], cfg.rounds_per_launch,
                                                                       ring) > 0)
          work = true;
    }
    if (work || !admitted.empty()) {
      Launch &l = L[(next_id - 1) % kDepth];
      l.id = next_id++;
      st = enqueue(l, admitted);
      if (st != LABS_OK) break;
      inflight.push_back((int)((l.id - 1) % kDepth));
      continue;
    }
    if (!inflight.empty()) {
      harvest_oldest();
      continue;
    }
    std::unique_lock<std::mutex> lock(mu);
    if (!stopping && pending.empty()) wake.wait_for(lock, std::chrono::milliseconds(20));
  }
  // device work must end before teardown; requests not finished end with a status
  for (int li : inflight) cudaEventSynchronize(L[li].ev1);
  fail_all(st != LABS_OK ? st : LABS_ESHUTDOWN);
}

extern "C" void labs_serve_cfg_init(labs_serve_cfg *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->mem_bytes = (size_t)8 << 30;
  c->max_active = 64;
  c->max_L = 301;
  c->max_walks = 2048;
  c->max_walk_len = 0;
  c->rounds_per_launch = 4;
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
      cfg.max_walk_len > (1 << 26) ||
      cfg.rounds_per_launch <= 0 || cfg.rounds_per_launch > 64 || cfg.block_threads < 32 ||
      cfg.block_threads > 256 || cfg.block_threads % 32 || cfg.mem_bytes < 2 * kAlign || cfg.walk_mode < 0 ||
      cfg.walk_mode > 2 || (cfg.walk_mode == 2 && cfg.max_walks > kWarpModeMaxWalks))
    return LABS_EINVAL;
  if (cfg.max_walk_len == 0) cfg.max_walk_len = 8 * ((cfg.max_L + 1) / 2);
  labs_server *sv = new (std::nothrow) labs_server();
  if (!sv) return LABS_ENOMEM;
  sv->cfg = cfg;
  auto fail = [&](labs_status e) {
    delete sv;
    return e;
  };
  if (cudaGetDevice(&sv->device) != cudaSuccess) return fail(LABS_ECUDA);
  const int n = cfg.max_active;
  const int Wmax = lag_words(cfg.max_L);
  const uint32_t ring = (uint32_t)(kRingFactor * cfg.rounds_per_launch);
  const uint32_t max_chunks = (uint32_t)((cfg.max_walks + 31) / 32);
  const size_t nrec = (size_t)n * ring;
  sv->warp_allowed = cfg.max_walks <= kWarpModeMaxWalks && cfg.walk_mode != 1;
  const uint32_t max_keys = sv->warp_allowed ? (uint32_t)cfg.max_walks : max_chunks;
  // what each class keeps resident in either mode (rates measured below)
  size_t tune_slots = 1;
  for (int W = 1; W <= Wmax; ++W) {
    ClassInfo ci;
    ci.resident[0] = batch_resident_lanes(W, cfg.block_threads, 1);
    ci.resident[1] = batch_resident_lanes(W, cfg.block_threads, 2);
    ci.resident[2] = batch_resident_warps(W, cfg.block_threads);
    if (ci.resident[0] <= 0 || ci.resident[1] <= 0 || ci.resident[2] <= 0) return fail(LABS_ECUDA);
    sv->cls.push_back(ci);
    tune_slots = std::max<size_t>(tune_slots, std::max({ci.resident[0] / 32, ci.resident[1] / 32, ci.resident[2]}));
  }
  sv->ring = ring;
  sv->slot_ticket.assign(n, 0);
  sv->slot_listed.assign(n, 0);
  sv->slot_draining.assign(n, 0);
  // fixed state: per slot, then the round records
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t o_probs = take(sizeof(BatchProblem) * n), o_base = take(sizeof(uint32_t) * n),
               o_ring = take(sizeof(uint32_t) * n), o_budget = take(sizeof(uint64_t) * n),
               o_target = take(sizeof(int64_t) * n), o_fin = take(sizeof(uint32_t) * n),
               o_done = take(sizeof(int32_t) * n), o_bestE = take(sizeof(int64_t) * n),
               o_key = take(sizeof(uint32_t) * kKeyWords * n), o_brnd = take(sizeof(int32_t) * n),
               o_bwalk = take(sizeof(int32_t) * n), o_evals = take(sizeof(unsigned long long) * n),
               o_planes = take(sizeof(unsigned long long) * n), o_rounds = take(sizeof(int32_t) * n),
               o_err = take(sizeof(int32_t)),
               o_rbest = take(sizeof(unsigned long long) * (nrec + 1)),
               o_revals = take(sizeof(unsigned long long) * (nrec + 1)),
               o_rplanes = take(sizeof(unsigned long long) * (nrec + 1)), o_rleft = take(sizeof(uint32_t) * (nrec + 1)),
               o_rround = take(sizeof(uint32_t) * (nrec + 1)), o_rshift = take(sizeof(uint32_t) * (nrec + 1)),
               o_rkbase = take(sizeof(unsigned long long) * (nrec + 1)),
               // the records' key slots, then those of the one record the mode timing uses
               o_rkeys = take(sizeof(uint32_t) * kKeyWords * (nrec * max_keys + tune_slots));
  char *fb = nullptr;
  if (cudaMalloc((void **)&fb, off) != cudaSuccess) return fail(LABS_ENOMEM);
  sv->fixed = fb;
  sv->fixed_bytes = off;
  if (cudaMemset(fb, 0, off) != cudaSuccess) return fail(LABS_ECUDA);
  sv->d_probs = reinterpret_cast<BatchProblem *>(fb + o_probs);
  sv->d_err = reinterpret_cast<int32_t *>(fb + o_err);
  ProblemState &ps = sv->ps;
  ps.rec_base = reinterpret_cast<uint32_t *>(fb + o_base);
  ps.ring = reinterpret_cast<uint32_t *>(fb + o_ring);
  ps.budget = reinterpret_cast<uint64_t *>(fb + o_budget);
  ps.target = reinterpret_cast<int64_t *>(fb + o_target);
  ps.fin = reinterpret_cast<uint32_t *>(fb + o_fin);
  ps.done = reinterpret_cast<int32_t *>(fb + o_done);
  ps.bestE = reinterpret_cast<int64_t *>(fb + o_bestE);
  ps.key = reinterpret_cast<uint32_t *>(fb + o_key);
  ps.best_round = reinterpret_cast<int32_t *>(fb + o_brnd);
  ps.best_walk = reinterpret_cast<int32_t *>(fb + o_bwalk);
  ps.evals = reinterpret_cast<unsigned long long *>(fb + o_evals);
  ps.planes = reinterpret_cast<unsigned long long *>(fb + o_planes);
  ps.rounds = reinterpret_cast<int32_t *>(fb + o_rounds);
  RoundRecords &rec = sv->rec;
  rec.best = reinterpret_cast<unsigned long long *>(fb + o_rbest);
  rec.evals = reinterpret_cast<unsigned long long *>(fb + o_revals);
  rec.planes = reinterpret_cast<unsigned long long *>(fb + o_rplanes);
  rec.left = reinterpret_cast<uint32_t *>(fb + o_rleft);
  rec.round = reinterpret_cast<uint32_t *>(fb + o_rround);
  rec.shift = reinterpret_cast<uint32_t *>(fb + o_rshift);
  rec.keys = reinterpret_cast<uint32_t *>(fb + o_rkeys);
  rec.key_base = reinterpret_cast<unsigned long long *>(fb + o_rkbase);
  sv->tune_record = (uint32_t)nrec;
  {
    std::vector<uint32_t> base(n), rng(n, ring);
    for (int i = 0; i < n; ++i) base[i] = (uint32_t)i * ring;
    std::vector<int32_t> done(n, 1);  // free slots count as finished
    std::vector<unsigned long long> kbase(nrec + 1);  // max_keys slots per record, then the timing record's
    for (size_t j = 0; j <= nrec; ++j) kbase[j] = (unsigned long long)j * max_keys;
    if (cudaMemcpy(fb + o_base, base.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(fb + o_ring, rng.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(fb + o_done, done.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(fb + o_rkbase, kbase.data(), sizeof(unsigned long long) * (nrec + 1), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(fb + o_rround, 0xFF, sizeof(uint32_t) * (nrec + 1)) != cudaSuccess)
      return fail(LABS_ECUDA);
  }
  sv->half_bytes = cfg.mem_bytes / 2 / kAlign * kAlign;
  if (cudaMalloc((void **)&sv->arena, cfg.mem_bytes) != cudaSuccess) return fail(LABS_ENOMEM);
  // the launches in flight: streams, events, arena halves, snapshots
  for (int d = 0; d < kDepth; ++d) {
    Launch &l = sv->L[d];
    l.arena = sv->arena + (size_t)d * sv->half_bytes;
    if (cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking) != cudaSuccess) return fail(LABS_ECUDA);
    for (int W = 1; W <= Wmax; ++W) {
      cudaStream_t x;
      cudaEvent_t e;
      if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return fail(LABS_ECUDA);
      l.cs.push_back(x);
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(LABS_ECUDA);
      l.cs_done.push_back(e);
    }
    if (cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&l.ev0) != cudaSuccess || cudaEventCreate(&l.ev1) != cudaSuccess)
      return fail(LABS_ECUDA);
    size_t so = 0;
    auto stake = [&](size_t bytes) {
      const size_t o = so;
      so = align_up(so + bytes);
      return o;
    };
    const size_t s_done = stake(sizeof(int32_t) * n), s_rounds = stake(sizeof(int32_t) * n),
                 s_bestE = stake(sizeof(int64_t) * n), s_evals = stake(sizeof(unsigned long long) * n),
                 s_planes = stake(sizeof(unsigned long long) * n), s_seq = stake((size_t)kSeqStride * n),
                 s_next = stake(sizeof(unsigned int) * Wmax), s_init = stake(sizeof(int32_t) * n),
                 s_run = stake(sizeof(unsigned long long)), s_err = stake(sizeof(int32_t));
    if (cudaMalloc((void **)&l.d_snap, so) != cudaSuccess) return fail(LABS_ENOMEM);
    if (cudaMallocHost((void **)&l.h_snap, so) != cudaSuccess) return fail(LABS_ENOMEM);
    if (cudaMemset(l.d_snap, 0, so) != cudaSuccess) return fail(LABS_ECUDA);
    sv->fixed_bytes += so;
    l.snap.done = reinterpret_cast<int32_t *>(l.d_snap + s_done);
    l.snap.rounds = reinterpret_cast<int32_t *>(l.d_snap + s_rounds);
    l.snap.bestE = reinterpret_cast<int64_t *>(l.d_snap + s_bestE);
    l.snap.evals = reinterpret_cast<unsigned long long *>(l.d_snap + s_evals);
    l.snap.planes = reinterpret_cast<unsigned long long *>(l.d_snap + s_planes);
    l.snap.seq = reinterpret_cast<int8_t *>(l.d_snap + s_seq);
    l.snap.stride = kSeqStride;
    l.task_next = reinterpret_cast<unsigned int *>(l.d_snap + s_next);
    l.snap.run_evals = reinterpret_cast<unsigned long long *>(l.d_snap + s_run);
    l.init_list = reinterpret_cast<int32_t *>(l.d_snap + s_init);
    l.snap_err = reinterpret_cast<int32_t *>(l.d_snap + s_err);
    l.snap_bytes = so;
  }
  if (cudaEventCreate(&sv->t_ref) != cudaSuccess) return fail(LABS_ECUDA);
  // the server's work starts after what the caller's stream has queued
  cudaStream_t first = cfg.stream ? (cudaStream_t)cfg.stream : nullptr;
  if (cudaEventRecord(sv->t_ref, first) != cudaSuccess) return fail(LABS_ECUDA);
  for (int d = 0; d < kDepth; ++d)
    if (cudaStreamWaitEvent(sv->L[d].s, sv->t_ref, 0) != cudaSuccess) return fail(LABS_ECUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(LABS_ECUDA);
  labs_status tst = sv->tune_modes();
  if (tst != LABS_OK) return fail(tst);
  for (auto &ci : sv->cls) ci.forced = cfg.walk_mode;
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
  if (p.L < LABS_L_MIN || p.L > LABS_L_MAX || !(p.L & 1) || p.walks < 1 || p.walk_len < 1 ||
      p.walk_len > (1 << 26) || p.step_budget < 1)
    return LABS_EINVAL;
  // requests that can never be admitted: above the server's limits, or a
  // launch over this request alone does not fit half the arena
  if (p.L > sv->cfg.max_L || p.walks > sv->cfg.max_walks || p.walk_len > sv->cfg.max_walk_len) return LABS_ENOMEM;
  {
    std::vector<Share> one{share_of(-1, p, (uint32_t)sv->cfg.rounds_per_launch)};
    if (carve_launch(one, sv->cls, sv->cfg.block_threads).total > sv->half_bytes) return LABS_ENOMEM;
  }
  auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
  if (!r) return LABS_ENOMEM;
  r->p = p;
  r->W = lag_words(p.L);
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
    out->plane_steps = r.planes;
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
  for (size_t i = 0; i < sv->slot_ticket.size(); ++i) act += sv->slot_ticket[i] != 0 && !sv->slot_draining[i];
  out->active = (uint64_t)act;
  out->evals = sv->evals_done;
  out->evals_run = sv->evals_run;
  out->launches = sv->launches;
  out->walk_launches = sv->walk_launches;
  out->busy_ms = sv->busy_ms;
  out->mem_used = sv->mem_used;
  out->mem_peak = sv->mem_peak;
  out->lane_launches = sv->mode_launches[0];
  out->lane_unrolled_launches = sv->mode_launches[1];
  out->warp_launches = sv->mode_launches[2];
  out->fixed_bytes = sv->fixed_bytes;
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
  delete sv;
  return LABS_OK;
}
