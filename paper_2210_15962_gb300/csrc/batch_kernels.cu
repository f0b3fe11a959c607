// Host-callable side of the persistent batched execution that is the same
// for every lag-word class: the dispatch to the per-class kernels
// (batch_class.cu), the post-launch finalization, the issue of round records,
// the reset of problems and the snapshot.
#include <climits>

#include "batch_device.cuh"

namespace psaw {

template <int W>
cudaError_t launch_batch_class(int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out, int max_blocks,
                               int variant);
template <int W>
int batch_resident_class(int block, int variant);
#define PSAW_BATCH_CLASS(W)                                                                                   \
  extern template cudaError_t launch_batch_class<W>(int, const BatchKernelParams &, cudaStream_t, int *, int, \
                                                    int);                                                     \
  extern template int batch_resident_class<W>(int, int);
PSAW_BATCH_CLASS(1)
PSAW_BATCH_CLASS(2)
PSAW_BATCH_CLASS(3)
PSAW_BATCH_CLASS(4)
PSAW_BATCH_CLASS(5)
PSAW_BATCH_CLASS(6)
PSAW_BATCH_CLASS(7)
PSAW_BATCH_CLASS(8)
#undef PSAW_BATCH_CLASS

static cudaError_t dispatch_launch(int W, int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out,
                                   int max_blocks, int variant) {
  if (block < 32 || block > kBatchMaxThreads || block % 32) return cudaErrorInvalidValue;
  switch (W) {
    case 1: return launch_batch_class<1>(block, p, s, grid_out, max_blocks, variant);
    case 2: return launch_batch_class<2>(block, p, s, grid_out, max_blocks, variant);
    case 3: return launch_batch_class<3>(block, p, s, grid_out, max_blocks, variant);
    case 4: return launch_batch_class<4>(block, p, s, grid_out, max_blocks, variant);
    case 5: return launch_batch_class<5>(block, p, s, grid_out, max_blocks, variant);
    case 6: return launch_batch_class<6>(block, p, s, grid_out, max_blocks, variant);
    case 7: return launch_batch_class<7>(block, p, s, grid_out, max_blocks, variant);
    case 8: return launch_batch_class<8>(block, p, s, grid_out, max_blocks, variant);
    default: return cudaErrorInvalidValue;
  }
}

static int dispatch_resident(int W, int block, int variant) {
  switch (W) {
    case 1: return batch_resident_class<1>(block, variant);
    case 2: return batch_resident_class<2>(block, variant);
    case 3: return batch_resident_class<3>(block, variant);
    case 4: return batch_resident_class<4>(block, variant);
    case 5: return batch_resident_class<5>(block, variant);
    case 6: return batch_resident_class<6>(block, variant);
    case 7: return batch_resident_class<7>(block, variant);
    case 8: return batch_resident_class<8>(block, variant);
    default: return 0;
  }
}

cudaError_t launch_batch(int W, int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out,
                         int max_blocks, int unroll) {
  return dispatch_launch(W, block, p, s, grid_out, max_blocks, unroll == 2 ? kBatchLaneUnroll2 : kBatchLane);
}

cudaError_t launch_batch_warp(int W, int block, const BatchKernelParams &p, cudaStream_t s, int max_blocks) {
  return dispatch_launch(W, block, p, s, nullptr, max_blocks, kBatchWarp);
}

int batch_resident_lanes(int W, int block, int unroll) {
  return dispatch_resident(W, block, unroll == 2 ? kBatchLaneUnroll2 : kBatchLane);
}
int batch_resident_warps(int W, int block) { return dispatch_resident(W, block, kBatchWarp); }

cudaError_t launch_batch_cta(int W, const BatchKernelParams &p, cudaStream_t s, int max_blocks) {
  return dispatch_launch(W, kWalkBlock, p, s, nullptr, max_blocks, kBatchCta);
}
int batch_resident_ctas(int W) { return dispatch_resident(W, kWalkBlock, kBatchCta); }

// After a launch: finalize what the in-kernel finalization left (normally
// nothing), one thread per listed problem.
__global__ void batch_finalize_kernel(const int32_t *problems, int n, const RoundRecords rec, const ProblemState ps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) try_finalize(rec, ps, problems[i]);
}

cudaError_t launch_batch_finalize(const int32_t *problems, int n, const RoundRecords &rec, const ProblemState &ps,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  batch_finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(problems, n, rec, ps);
  return cudaGetLastError();
}

// New rounds in their records: the accumulators and the chunk count first,
// then (after a fence) the round number, which makes the record the round's.
__global__ void issue_records_kernel(const RecordInit *list, int n, const RoundRecords rec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RecordInit ri = list[i];
  rec.best[ri.rec] = ~0ull;
  rec.evals[ri.rec] = 0;
  rec.planes[ri.rec] = 0;
  rec.left[ri.rec] = ri.chunks;
  rec.shift[ri.rec] = ri.shift;
  __threadfence();
  rec.round[ri.rec] = ri.round;
}

cudaError_t launch_issue_records(const RecordInit *list, int n, const RoundRecords &rec, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  issue_records_kernel<<<(n + 127) / 128, 128, 0, s>>>(list, n, rec);
  return cudaGetLastError();
}

// A problem starting afresh: its records hold no round, then its state.
__global__ void init_problems_state_kernel(const int32_t *problems, int n, const RoundRecords rec,
                                           const ProblemState ps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = problems[i];
  for (uint32_t k = 0; k < ps.ring[p]; ++k) rec.round[ps.rec_base[p] + k] = ~0u;
  __threadfence();
  ps.fin[p] = 0;
  ps.bestE[p] = INT64_MAX;
  ps.evals[p] = 0;
  ps.planes[p] = 0;
  ps.rounds[p] = 0;
  ps.best_round[p] = -1;
  ps.best_walk[p] = -1;
  for (int k = 0; k < kKeyWords; ++k) ps.key[(size_t)p * kKeyWords + k] = 0u;
  __threadfence();
  ps.done[p] = 0;
}

cudaError_t launch_init_problems_state(const int32_t *problems, int n, const RoundRecords &rec,
                                       const ProblemState &ps, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  init_problems_state_kernel<<<(n + 127) / 128, 128, 0, s>>>(problems, n, rec, ps);
  return cudaGetLastError();
}

// One block per listed problem: its state, read after its done flag (the
// finalizer writes the flag last, after a fence, so a finished problem's state
// is complete), and the Eq. 2 expansion of its best key when it is finished.
// Block 0 also sums the evaluations of the listed records.
__global__ void snapshot_kernel(const int32_t *problems, int n, const BatchProblem *probs, const ProblemState ps,
                                const uint32_t *recs, int n_recs, const RoundRecords rec, const Snapshot out) {
  const int p = problems[blockIdx.x];
  __shared__ int32_t fin_done;
  if (threadIdx.x == 0) {
    const int32_t d = load_volatile(ps.done + p);
    __threadfence();
    out.done[p] = d;
    out.rounds[p] = __ldcg(ps.rounds + p);
    out.bestE[p] = (int64_t)__ldcg(reinterpret_cast<const long long *>(ps.bestE) + p);
    out.evals[p] = __ldcg(ps.evals + p);
    out.planes[p] = __ldcg(ps.planes + p);
    fin_done = d;
  }
  __syncthreads();
  if (fin_done) {
    const int L = probs[p].L;
    uint32_t key[kKeyWords];
    for (int k = 0; k < kKeyWords; ++k) key[k] = __ldcg(ps.key + (size_t)p * kKeyWords + k);
    for (int a = threadIdx.x; a < L; a += blockDim.x)
      out.seq[(size_t)p * out.stride + a] = sequence_bit(key, L, a, false) ? (int8_t)-1 : (int8_t)1;
  }
  if (blockIdx.x == 0 && out.run_evals) {
    unsigned long long sum = 0;
    for (int i = threadIdx.x; i < n_recs; i += blockDim.x) sum += __ldcg(rec.evals + recs[i]);
    if (sum) atomicAdd(out.run_evals, sum);
  }
}

cudaError_t launch_snapshot(const int32_t *problems, int n, const BatchProblem *probs, const ProblemState &ps,
                            const uint32_t *recs, int n_recs, const RoundRecords &rec, const Snapshot &out,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  snapshot_kernel<<<n, 128, 0, s>>>(problems, n, probs, ps, recs, n_recs, rec, out);
  return cudaGetLastError();
}

}  // namespace psaw
