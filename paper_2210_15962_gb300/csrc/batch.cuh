// Persistent batched execution of many problems of uneven L (Eq. 4 rounds of
// Algorithm 2 walks for several independent instances at once), shared by the
// batch entry points and the serving loop.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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

// one warp task: 32 walks (chunk) of one round of one problem
struct BatchTask {
  uint32_t problem, round, chunk, slot;
};

struct BatchKernelParams {
  const BatchProblem *probs;
  const BatchTask *tasks;
  uint32_t n_tasks;
  unsigned int *task_next;         // dynamic task counter
  uint64_t *pool;                  // visited tables, one per resident lane
  size_t pool_words;               // 64-bit words per lane
  unsigned long long *slot_best;   // per (problem, round) slot: (E << 32) | walk, atomicMin
  unsigned long long *slot_evals;  // per slot: neighbour evaluations
  uint32_t *slot_keys;             // [slot][chunk][kKeyWords]: best key of each chunk
  uint32_t max_chunks;
  const int32_t *done;             // per problem, nonzero = skip its tasks
  uint32_t mul_one, mul_two, mul_four, mul_h31, mul_h30;
  unsigned long long *plane_steps;
  int32_t *err;
};

struct BatchFinalizeParams {
  int32_t n_problems;
  const uint32_t *first_slot;  // per problem: its first slot in this launch
  const uint32_t *n_slots;     // per problem: rounds it ran in this launch (in round order)
  const uint32_t *slot_round;  // per slot: round index
  const unsigned long long *slot_best;
  const unsigned long long *slot_evals;
  const uint32_t *slot_keys;
  uint32_t max_chunks;
  const uint64_t *budget;
  const int64_t *target;
  int32_t *done;
  int64_t *bestE;
  uint32_t *key;  // [problem][kKeyWords]
  int32_t *best_round, *best_walk;
  unsigned long long *evals;
  int32_t *rounds;
};

// Launch the persistent kernel for lag-word class W with `block` threads per
// block and as many blocks as fit on the device at once.
cudaError_t launch_batch(int W, int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out);
// Lanes the persistent kernel of class W keeps resident with `block` threads per block.
int batch_resident_lanes(int W, int block);
cudaError_t launch_batch_finalize(const BatchFinalizeParams &f, cudaStream_t s);
cudaError_t launch_init_slots(const int32_t *slots, int n, int64_t *bestE, unsigned long long *evals, int32_t *done,
                              int32_t *rounds, int32_t *best_round, int32_t *best_walk, uint32_t *key, cudaStream_t s);

}  // namespace psaw
