// Persistent batched execution of many problems of uneven L (Eq. 4 rounds of
// Algorithm 2 walks for several independent instances at once), shared by the
// batch entry points and the serving loop.
//
// Work unit: a task = 32 walks (one chunk) of one round of one problem.  Every
// issued (problem, round) has a round record in the problem's ring of records
// (record rec_base[p] + round % ring[p]); the warps that run its chunks add
// their evaluations and digit planes, atomicMin their best (E, walk) and
// publish their chunk's best key into it, and count the chunk done.  The warp
// that finishes a round's last chunk finalizes, in round order, every complete
// round of that problem (Algorithm 1: strict best, earliest round and lowest
// walk on ties, stop at the budget or the target), so a problem is marked
// done on the device as soon as its stopping round is final and the tasks of
// its later rounds, issued speculatively, are skipped when a warp takes them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <tuple>
#include <vector>

#include "walk_kernels.cuh"

namespace psaw {

// one problem as the device sees it
struct BatchProblem {
  int32_t L, W, walk_len, walks;
  uint32_t cap;  // visited-table slots of this problem's walks
  int32_t kw64;
  uint64_t seed;
};

// one warp task: 32 walks (chunk) of one round of one problem, or in warp
// mode one walk (chunk = the walk's index), and the round's record
struct BatchTask {
  uint32_t problem, round, chunk, rec;
};

// The round records (all problems' rings, one array per field).
struct RoundRecords {
  unsigned long long *best;    // (E << 32) | walk, atomicMin; ~0 = none yet
  unsigned long long *evals;   // neighbour evaluations of the round
  unsigned long long *planes;  // digit planes summed over the round's walk steps
  uint32_t *left;              // chunks not finished yet
  uint32_t *round;             // the round the record holds (~0 = none)
  uint32_t *shift;             // key slot of walk w = w >> shift: 5 (a slot per chunk) or 0 (per walk)
  const unsigned long long *key_base;  // per record: its first key slot
  uint32_t *keys;              // [slot][kKeyWords]: best key of each chunk or walk of each record
};

// Per-problem state of Algorithm 1, kept across the problem's launches.
struct ProblemState {
  const uint32_t *rec_base, *ring;  // the problem's records: rec_base[p] .. + ring[p] - 1
  const uint64_t *budget;
  const int64_t *target;
  uint32_t *fin;  // (next round to finalize) << 1 | lock bit
  int32_t *done;  // 1 once the budget or target stopped the problem
  int64_t *bestE;
  uint32_t *key;  // [problem][kKeyWords]
  int32_t *best_round, *best_walk;
  unsigned long long *evals, *planes;  // over the finalized rounds
  int32_t *rounds;                     // rounds finalized
};

struct BatchKernelParams {
  const BatchProblem *probs;
  const BatchTask *tasks;
  uint32_t n_tasks;
  unsigned int *task_next;  // dynamic task counter
  uint64_t *pool;           // visited tables, one per lane of the grid
  size_t pool_words;        // 64-bit words per lane
  RoundRecords rec;
  ProblemState ps;
  uint32_t mul_one, mul_two, mul_four, mul_h31, mul_h30;
  int32_t *err;
};

// A record about to hold `round` of a problem, which `chunks` tasks run
// (chunks of 32 walks, key shift 5; or single walks in warp mode, shift 0).
struct RecordInit {
  uint32_t rec, round, chunks, shift;
};

// A task with its place in a launch's order.  Problems with a target run the
// rounds of a launch layer by layer (layer = the round's index in the launch:
// round k of every such problem before round k + 1 of any), so a round that
// reaches the target stops the problem before its later rounds start; inside a
// layer, and for problems without a target (whose every round is needed, all
// in layer 0), the longest tasks go first so that the launch's tail is short.
struct PlannedTask {
  uint32_t layer;
  double cost;  // relative duration of the task
  BatchTask t;
};

inline void order_tasks(std::vector<PlannedTask> &v) {
  std::stable_sort(v.begin(), v.end(), [](const PlannedTask &x, const PlannedTask &y) {
    if (x.layer != y.layer) return x.layer < y.layer;
    if (x.cost != y.cost) return x.cost > y.cost;
    return std::tie(x.t.round, x.t.problem, x.t.chunk) < std::tie(y.t.round, y.t.problem, y.t.chunk);
  });
}

// relative duration of one task (32 walks): steps x flips x lag words
inline double batch_task_cost(int L, int walk_len) {
  return (double)walk_len * (double)((L + 1) / 2) * (double)lag_words(L);
}

// Reset the listed records for their new rounds (before any of their tasks run).
cudaError_t launch_issue_records(const RecordInit *list, int n, const RoundRecords &rec, cudaStream_t s);
// Kernel variants of a class: one walk per lane, the same with the scan's
// flip loop unrolled twice, one walk per warp, and one walk per CTA.
constexpr int kBatchLane = 0, kBatchWarp = 1, kBatchLaneUnroll2 = 2, kBatchCta = 3;

// Launch the persistent kernel for lag-word class W with `block` threads per
// block and as many blocks as fit on the device at once, at most max_blocks
// when max_blocks > 0 (the pool must hold grid * block lanes); unroll 1 or 2
// unrolls the scan's flip loop.
cudaError_t launch_batch(int W, int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out,
                         int max_blocks = 0, int unroll = 1);
// Lanes the persistent kernel of class W keeps resident with `block` threads per block.
int batch_resident_lanes(int W, int block, int unroll = 1);
// Warp mode (one walk per warp, tasks of one walk; the pool holds one table
// per warp of the grid): the launch, and the warps it keeps resident.
cudaError_t launch_batch_warp(int W, int block, const BatchKernelParams &p, cudaStream_t s, int max_blocks = 0);
int batch_resident_warps(int W, int block);
// CTA mode (one walk per CTA of 128 threads, tasks of one walk; the pool holds
// one table per CTA of the grid): the launch, and the CTAs it keeps resident.
cudaError_t launch_batch_cta(int W, const BatchKernelParams &p, cudaStream_t s, int max_blocks = 0);
int batch_resident_ctas(int W);
// Finalize, in round order, the complete rounds of the listed problems (those
// the in-kernel finalization left, normally none).
cudaError_t launch_batch_finalize(const int32_t *problems, int n, const RoundRecords &rec, const ProblemState &ps,
                                  cudaStream_t s);
// Start the listed problems afresh: no round finalized, no best, not done,
// their records emptied.
cudaError_t launch_init_problems_state(const int32_t *problems, int n, const RoundRecords &rec,
                                       const ProblemState &ps, cudaStream_t s);
// Where launch_snapshot copies the state of the listed problems (done,
// rounds, best E, evaluations and planes at the problem's index, and the best
// sequence, Eq. 2, of each finished one at seq + p * stride), and the counter
// to which it adds the evaluations of the listed records.
struct Snapshot {
  int32_t *done, *rounds;
  int64_t *bestE;
  unsigned long long *evals, *planes;
  int8_t *seq;
  int stride;
  unsigned long long *run_evals;
};
cudaError_t launch_snapshot(const int32_t *problems, int n, const BatchProblem *probs, const ProblemState &ps,
                            const uint32_t *recs, int n_recs, const RoundRecords &rec, const Snapshot &out,
                            cudaStream_t s);

}  // namespace psaw
