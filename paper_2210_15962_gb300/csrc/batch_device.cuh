// Device side of the persistent batched execution (batch.cuh): the task
// loops of lane mode (a warp takes tasks of 32 walks, one walk per lane) and
// warp mode (a warp takes tasks of one walk, its lanes split the flips), and
// the in-kernel round finalization they share with the post-launch pass.
#pragma once
#include "batch.cuh"
#include "walk_cta.cuh"
#include "walk_device.cuh"
#include "walk_warp.cuh"

namespace psaw {

constexpr int kBatchMaxThreads = 256;

// Widest lag-word class whose scan runs through pattern-specialised loops: the
// classes' persistent kernels run side by side, so their code shares the SMs'
// instruction caches and is kept smaller than in the per-round kernel
// (measured on the serving mix, one class at a time: specialised loops gain
// 12% at three words and lose 20% at four).
constexpr int kBatchPatternMaxWords = 3;

// register budget per thread of each class (the task loop keeps more state
// live than the per-round kernel).  Measured one class at a time (38 to 76
// problems of 2048 walks, autotuned shapes): two words run 6-10% faster at 96
// than at 112 (80: 4-9%), five words 4% faster at 168 than at 208; three
// words lose 5-9% at 102, and six to eight words, which also fit 168 without
// spilling, run 1-15% slower there than unbounded.  Tighter budgets that
// spill measured slower.
template <int W>
struct MaxRegsFor {
  static constexpr int value = W == 1 ? 104 : (W == 2 ? 96 : (W <= 4 ? 128 : (W == 5 ? 168 : 255)));
};

// shared memory words of one warp: mask table, then (W + 2) parked words per lane
template <int W>
constexpr int kBatchWarpWords = MaskTable<W>::kWords + (W + 2) * 32;
// in warp mode (one walk per warp): mask table, then the walk's shared words,
// rounded to 16 bytes so that every warp's mask table stays 16-byte aligned
template <int W>
constexpr int kBatchWalkWarpWords = (MaskTable<W>::kWords + WarpWalkSmem<W>::kWords + 3) / 4 * 4;
// in CTA mode (one walk per CTA of kWalkBlock threads): the mask table, the
// walk's CtaWalkSmem words, then the task index and its problem's stop flag as
// thread 0 read them
template <int W>
constexpr int kBatchWalkCtaWords = MaskTable<W>::kWords + CtaWalkSmem<W>::kWords + 2;

__device__ __forceinline__ uint32_t load_volatile(const uint32_t *x) { return *(const volatile uint32_t *)x; }
__device__ __forceinline__ int32_t load_volatile(const int32_t *x) { return *(const volatile int32_t *)x; }

__device__ __forceinline__ uint32_t record_of(const ProblemState &ps, int p, uint32_t round) {
  return ps.rec_base[p] + round % ps.ring[p];
}

// Algorithm 1's update with round r of problem p (its record complete, the
// caller holding p's finalization lock): add the round's evaluations, keep
// the strict best (so the earliest round wins ties, and inside a round the
// lowest walk through the atomicMin key), and stop at the budget or the
// target.  Returns true when the problem stops here.  Reads bypass L1: the
// record and the state were written by other SMs.
inline __device__ bool finalize_round(const RoundRecords &rec, const ProblemState &ps, int p, uint32_t r) {
  const uint32_t j = record_of(ps, p, r);
  const unsigned long long ev = __ldcg(ps.evals + p) + __ldcg(rec.evals + j);
  ps.evals[p] = ev;
  ps.planes[p] = __ldcg(ps.planes + p) + __ldcg(rec.planes + j);
  const unsigned long long rb = __ldcg(rec.best + j);
  long long best = __ldcg(reinterpret_cast<const long long *>(ps.bestE) + p);
  if (rb != ~0ull) {
    const long long E = (long long)(rb >> 32);
    const uint32_t w = (uint32_t)(rb & 0xFFFFFFFFu);
    if (E < best) {
      best = E;
      ps.bestE[p] = E;
      // the round's key slots: one per chunk of 32 walks, or one per walk (warp mode)
      const uint32_t *src = rec.keys + (__ldcg(rec.key_base + j) + (w >> __ldcg(rec.shift + j))) * kKeyWords;
      for (int i = 0; i < kKeyWords; ++i) ps.key[(size_t)p * kKeyWords + i] = __ldcg(src + i);
      ps.best_round[p] = (int32_t)r;
      ps.best_walk[p] = (int32_t)w;
    }
  }
  ps.rounds[p] = (int32_t)r + 1;
  if (ev >= ps.budget[p] || (ps.target[p] >= 0 && best <= ps.target[p])) {
    __threadfence();  // the state above is visible before `done`
    ps.done[p] = 1;
    return true;
  }
  return false;
}

// Finalize the complete rounds of problem p that are next in round order.
// Called by one thread after it completed a chunk of one of p's rounds (or by
// the post-launch pass).  fin[p] = (next round) << 1 | lock: whoever takes the
// lock finalizes, unlocks, then looks again, so a round that completes while
// another is being finalized is never left behind (the completer's count
// update and the finalizer's unlock are each followed by a full fence before
// each reads the other's word).  A record is the next round's only if it holds
// that round (records are reused round after round), read before its count.
// `done` is read again under the lock: a thread that saw the problem running
// may take the lock right after the round that stopped it was finalized (the
// stopping finalizer writes `done` before it unlocks), and must not add the
// next round.
inline __device__ void try_finalize(const RoundRecords &rec, const ProblemState &ps, int p) {
  for (;;) {
    if (load_volatile(ps.done + p)) return;
    __threadfence();
    const uint32_t st = load_volatile(ps.fin + p);
    if (st & 1u) return;  // another thread is finalizing; it looks at the next round after
    const uint32_t r = st >> 1;
    const uint32_t j = record_of(ps, p, r);
    if (load_volatile(rec.round + j) != r) return;  // round r not issued yet
    __threadfence();
    if (load_volatile(rec.left + j) != 0u) return;  // round r not complete yet
    if (atomicCAS(ps.fin + p, st, st | 1u) != st) continue;
    __threadfence();
    if (load_volatile(ps.done + p)) {  // stopped by the round before r
      atomicExch(ps.fin + p, st);
      return;
    }
    const bool stop = finalize_round(rec, ps, p, r);
    __threadfence();
    atomicExch(ps.fin + p, (r + 1u) << 1);
    __threadfence();
    if (stop) return;
  }
}

template <int W, int U>
__global__ void __launch_bounds__(kBatchMaxThreads) __maxnreg__(MaxRegsFor<W>::value)
    batch_kernel(const BatchKernelParams p) {
  constexpr int T = PlanesFor<W>::value;
  constexpr int NS = W + 1;
  const int lane = threadIdx.x & 31;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t *table = p.pool + gtid * p.pool_words;
  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  // each warp's valid-lag mask table (refilled when its task's L changes) and
  // its lanes' parked best pivots
  extern __shared__ __align__(16) uint32_t batch_smem[];
  uint32_t *mask_rows = batch_smem + (size_t)(threadIdx.x >> 5) * kBatchWarpWords<W>;
  uint32_t *best_park = mask_rows + MaskTable<W>::kWords + lane;
  int rows_L = 0;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(p.task_next, 1u);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= p.n_tasks) break;
    const BatchTask task = p.tasks[t];
    // a problem stopped by an earlier round (finalized in an earlier launch or
    // by a warp of this one) needs none of its later rounds: skip them
    if (load_volatile(p.ps.done + task.problem)) continue;
    const BatchProblem pr = p.probs[task.problem];
    const uint32_t walk = task.chunk * 32u + (uint32_t)lane;
    const bool active = walk < (uint32_t)pr.walks;
    clear_tables_warp(table, (size_t)pr.cap * (size_t)pr.kw64, active);
    const Geometry g = make_geometry(pr.L, T);
    if (pr.L != rows_L) {  // warp-uniform: every lane took the same task
      fill_mask_rows<W>(g, mask_rows, lane, 32);
      __syncwarp();
      rows_L = pr.L;
    }
    unsigned long long packed = ~0ull, planes = 0;
    uint32_t evals = 0;
    WalkOut<NS> o;
    if (active) {
      run_walk<W, T, kTopK, kBatchPatternMaxWords, U>(g, mu, mask_rows, best_park, 32, pr.seed, walk, task.round,
                                                      pr.walk_len, table, pr.cap, pr.kw64, 0, nullptr, p.err, o);
      packed = ((unsigned long long)(uint32_t)o.bestE << 32) | walk;
      evals = (uint32_t)g.D * (uint32_t)(o.moves + o.stuck);
      planes = o.planes;
    }
    // the chunk's best (lowest E, then lowest walk) publishes its key
    unsigned long long m = packed;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xFFFFFFFFu, m, off);
      m = v < m ? v : m;
      planes += __shfl_xor_sync(0xFFFFFFFFu, planes, off);
    }
    if (active && packed == m) {
      uint32_t *k = p.rec.keys + (p.rec.key_base[task.rec] + task.chunk) * kKeyWords;
#pragma unroll
      for (int w = 0; w < kKeyWords; ++w) k[w] = w < NS ? o.best_key[w] : 0u;
    }
    const uint32_t ev = __reduce_add_sync(0xFFFFFFFFu, evals);
    if (lane == 0) {
      atomicMin(&p.rec.best[task.rec], m);
      atomicAdd(&p.rec.evals[task.rec], (unsigned long long)ev);
      atomicAdd(&p.rec.planes[task.rec], planes);
    }
    // every lane's results are visible device-wide before the chunk counts as
    // finished; the warp that finishes a round's last chunk finalizes it
    __threadfence();
    __syncwarp();
    if (lane == 0 && atomicSub(&p.rec.left[task.rec], 1u) == 1u) {
      __threadfence();
      try_finalize(p.rec, p.ps, (int)task.problem);
    }
    __syncwarp();
  }
}

// Warp mode: every warp takes tasks of one walk (task.chunk = the walk's
// index) and runs the walk with its 32 lanes splitting the flips
// (run_walk_warp); one visited table per warp.  The walk publishes its best
// key in its own key slot of the round's record.
template <int W>
__global__ void __launch_bounds__(kBatchMaxThreads) __maxnreg__(MaxRegsFor<W>::value)
    batch_kernel_warp(const BatchKernelParams p) {
  constexpr int T = PlanesFor<W>::value;
  constexpr int NS = W + 1;
  const int lane = threadIdx.x & 31;
  const size_t gwarp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t *table = p.pool + gwarp * p.pool_words;
  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  extern __shared__ __align__(16) uint32_t batch_smem[];
  uint32_t *mask_rows = batch_smem + (size_t)(threadIdx.x >> 5) * kBatchWalkWarpWords<W>;
  uint32_t *wsm = mask_rows + MaskTable<W>::kWords;
  int rows_L = 0;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(p.task_next, 1u);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= p.n_tasks) break;
    const BatchTask task = p.tasks[t];
    if (load_volatile(p.ps.done + task.problem)) continue;
    const BatchProblem pr = p.probs[task.problem];
    const uint32_t walk = task.chunk;
    const size_t words = (size_t)pr.cap * (size_t)pr.kw64;  // even: cap >= 64
    uint4 *t4 = reinterpret_cast<uint4 *>(table);
    for (size_t i = (size_t)lane; i < words / 2; i += 32) t4[i] = make_uint4(0u, 0u, 0u, 0u);
    const Geometry g = make_geometry(pr.L, T);
    if (pr.L != rows_L) {
      fill_mask_rows<W>(g, mask_rows, lane, 32);
      rows_L = pr.L;
    }
    __syncwarp();
    WalkOut<NS> o;
    run_walk_warp<W, T, kTopK>(g, mu, mask_rows, wsm, pr.seed, walk, task.round, pr.walk_len, table, pr.cap,
                               pr.kw64, 0, nullptr, p.err, o);
    if (lane == 0) {
      uint32_t *k = p.rec.keys + (p.rec.key_base[task.rec] + walk) * kKeyWords;
#pragma unroll
      for (int w = 0; w < kKeyWords; ++w) k[w] = w < NS ? o.best_key[w] : 0u;
      atomicMin(&p.rec.best[task.rec], ((unsigned long long)(uint32_t)o.bestE << 32) | walk);
      atomicAdd(&p.rec.evals[task.rec], (unsigned long long)g.D * (unsigned long long)(o.moves + o.stuck));
      atomicAdd(&p.rec.planes[task.rec], (unsigned long long)o.planes);
      __threadfence();
      if (atomicSub(&p.rec.left[task.rec], 1u) == 1u) {
        __threadfence();
        try_finalize(p.rec, p.ps, (int)task.problem);
      }
    }
    __syncwarp();
  }
}

// CTA mode: every CTA of kWalkBlock threads takes tasks of one walk
// (task.chunk = the walk's index) and runs the walk with its threads splitting
// the flips (run_walk_cta); one visited table per CTA.  Thread 0 takes the
// task and reads its problem's stop flag for the whole block, so every thread
// takes the same branches; the walk publishes its best key in its own key slot
// of the round's record, as in warp mode.
template <int W>
__global__ void __launch_bounds__(kWalkBlock) __maxnreg__(MaxRegsFor<W>::value)
    batch_kernel_cta(const BatchKernelParams p) {
  constexpr int T = PlanesFor<W>::value;
  constexpr int NS = W + 1;
  const int tid = threadIdx.x;
  uint64_t *table = p.pool + (size_t)blockIdx.x * p.pool_words;
  const Muls mu{p.mul_one, p.mul_two, p.mul_four, p.mul_h31, p.mul_h30};
  extern __shared__ __align__(16) uint32_t batch_smem[];
  uint32_t *mask_rows = batch_smem;
  uint32_t *csm = mask_rows + MaskTable<W>::kWords;
  uint32_t *task_word = csm + CtaWalkSmem<W>::kWords;  // [0] task index, [1] its problem's stop flag
  int rows_L = 0;
  for (;;) {
    if (tid == 0) {
      const uint32_t t = atomicAdd(p.task_next, 1u);
      task_word[0] = t;
      task_word[1] = t < p.n_tasks ? (uint32_t)load_volatile(p.ps.done + p.tasks[t].problem) : 0u;
    }
    __syncthreads();
    const uint32_t t = task_word[0];
    const bool skip = task_word[1] != 0u;
    __syncthreads();  // every thread has read the task before thread 0 takes the next
    if (t >= p.n_tasks) break;
    if (skip) continue;  // a problem stopped by an earlier round needs none of its later rounds
    const BatchTask task = p.tasks[t];
    const BatchProblem pr = p.probs[task.problem];
    const uint32_t walk = task.chunk;
    const size_t words = (size_t)pr.cap * (size_t)pr.kw64;  // even: cap >= 64
    uint4 *t4 = reinterpret_cast<uint4 *>(table);
    for (size_t i = (size_t)tid; i < words / 2; i += kWalkBlock) t4[i] = make_uint4(0u, 0u, 0u, 0u);
    const Geometry g = make_geometry(pr.L, T);
    if (pr.L != rows_L) {  // block-uniform: every thread read the same task
      fill_mask_rows<W>(g, mask_rows, tid, kWalkBlock);
      rows_L = pr.L;
    }
    __syncthreads();  // the zeroed table and the mask table are visible to the block
    WalkOut<NS> o;
    run_walk_cta<W, T, kTopK>(g, mu, mask_rows, csm, pr.seed, walk, task.round, pr.walk_len, table, pr.cap,
                              pr.kw64, 0, nullptr, p.err, o);
    if (tid == 0) {
      uint32_t *k = p.rec.keys + (p.rec.key_base[task.rec] + walk) * kKeyWords;
#pragma unroll
      for (int w = 0; w < kKeyWords; ++w) k[w] = w < NS ? o.best_key[w] : 0u;
      atomicMin(&p.rec.best[task.rec], ((unsigned long long)(uint32_t)o.bestE << 32) | walk);
      atomicAdd(&p.rec.evals[task.rec], (unsigned long long)g.D * (unsigned long long)(o.moves + o.stuck));
      atomicAdd(&p.rec.planes[task.rec], (unsigned long long)o.planes);
      __threadfence();
      if (atomicSub(&p.rec.left[task.rec], 1u) == 1u) {
        __threadfence();
        try_finalize(p.rec, p.ps, (int)task.problem);
      }
    }
  }
}

}  // namespace psaw
