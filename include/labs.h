/*
 * labs.h -- C ABI of a GB300 (sm_103a) solver for the skew-symmetric
 * Low-Autocorrelation Binary Sequences problem by parallel contiguous
 * self-avoiding walks, after Bošković, Herzog and Brest, "Parallel
 * Self-Avoiding Walks for a Low-Autocorrelation Binary Sequences Problem"
 * (arXiv 2210.15962).
 *
 * Problem (Eq. 1): for S = (s_1..s_L), s_i in {+1,-1},
 *     C_k = sum_{i=1}^{L-k} s_i s_{i+k},  E = sum_{k=1}^{L-1} C_k^2,  F = L^2 / (2E).
 * Search space (Eq. 2): odd L, D = (L+1)/2 free values s_1..s_D, and
 *     s_{D+i} = (-1)^i s_{D-i}, i = 1..D-1.
 * Walk (Eq. 3, Algorithm 2): from a random pivot P_1, each step evaluates all
 * D neighbours (flip s_j and its mirror s_{L+1-j}) with an incremental update
 * of the C_k, moves to the lowest-energy neighbour that is not an earlier
 * pivot of the same walk (lowest j on ties), and records the walk's best.
 * Rounds (Eq. 4, Algorithm 1): every round runs many independent walks; the
 * problem's best is kept across rounds until a neighbour-evaluation budget
 * (or a target energy) is reached.
 *
 * Conventions shared by every entry point:
 *   - L is odd with LABS_L_MIN <= L <= LABS_L_MAX, otherwise LABS_EINVAL;
 *   - sequences are int8 arrays of +1/-1 of length L (s_1 first);
 *   - the random first pivot of walk w in round r of the problem seeded by
 *     `seed` uses Philox4x32-10 with key (seed & 0xffffffff, seed >> 32) and
 *     counter (w, r, b, 0); free value j takes bit j%32 of word (j/32)%4 of
 *     block b = j/128, bit 1 meaning -1;
 *   - one "neighbour evaluation" is one of the D flips examined at a step;
 *     a walk that finds all neighbours visited stops ("stuck") and its last
 *     scan counts as D evaluations;
 *   - a round always completes; rounds continue while the evaluations done
 *     are below step_budget and the best energy is above the target;
 *   - all buffers are caller-owned unless stated; no call keeps a pointer to
 *     a caller buffer after it returns, except a server (labs_serve_*),
 *     which owns its own memory;
 *   - no C++ exception crosses this interface; every call returns a status.
 *
 * Everything a call computes runs in this library's CUDA kernels on the
 * current CUDA device.  There is no CPU fallback: without a usable GPU the
 * calls return LABS_ECUDA.
 */
#ifndef LABS_H_
#define LABS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t labs_status;

#define LABS_OK 0
#define LABS_PENDING 1      /* labs_serve_poll: request not finished yet */
#define LABS_EINVAL (-1)    /* bad argument (L, sizes, null pointers, non +-1 values) */
#define LABS_ENOMEM (-2)    /* device memory could not be obtained or is too small */
#define LABS_ECUDA (-3)     /* a CUDA call failed (no device, launch error, ...) */
#define LABS_ETIMEOUT (-4)  /* a bounded wait expired */
#define LABS_EOVERFLOW (-5) /* a visited table ran out of slots (cannot happen with the sizes used) */
#define LABS_ENOTFOUND (-6) /* unknown server ticket */
#define LABS_ECHECK (-7)    /* the debug recheck found incremental and full energies different */
#define LABS_ESHUTDOWN (-8) /* server is shutting down */

#define LABS_L_MIN 5
#define LABS_L_MAX 511
/* lengths accepted by the full-search-space functions (labs_walks_full, ...) */
#define LABS_FULL_L_MIN 3
#define LABS_FULL_L_MAX 256

/* Options of labs_walks.  Zero-initialise (or call labs_opts_init), then set
 * what you need. */
typedef struct labs_opts {
  void *stream;           /* cudaStream_t to run on; NULL = legacy default stream */
  int32_t device_buffers; /* 0: seeds, best_seq, best_E are host pointers;
                             1: they are device pointers (stream-ordered, no
                                host copies of inputs or outputs) */
  int32_t recheck_every;  /* 0 = off; n > 0: every n steps each walk recomputes all
                             C_k and E with XOR+popc (Eq. 1) and compares them with its
                             incremental state; a mismatch makes the call return LABS_ECHECK */
  int64_t target_E;       /* stop a problem after the first round whose best E <= target_E;
                             < 0 = no target.  Set to -1 by labs_opts_init. */
  int32_t max_rounds;     /* 0 = no limit; else stop every problem after this many rounds */
  int32_t kernel;         /* neighbourhood evaluation: 0 = the library's choice (1, 3 or, for
                             launches of at most 16 walks per SM, 4: whichever ran a short
                             sample round of the same launch size faster; timed once per
                             process per lag-word class and launch size by the first call
                             with walks of >= 256 steps; a call of shorter walks times a
                             sample of its own),
                             1 = full scan, one lane per walk (every neighbour from the
                                 correlations each step),
                             2 = incremental (stored neighbour deltas updated after each move),
                             3 = full scan, one warp per walk (the lanes split the D flips),
                             4 = full scan, one CTA of 128 threads per walk (its threads split
                                 the D flips; the paper's block per walk, Algorithm 2);
                             all give the same results; other values: LABS_EINVAL (the full
                             search space takes 0 and 1 only) */
  void *workspace;        /* optional device scratch of workspace_bytes bytes (e.g. from
                             PyTorch); NULL = the library allocates and frees it itself */
  size_t workspace_bytes;
  uint64_t *evals_per_seed;  /* optional host (or device, if device_buffers) [n_seeds] out */
  int32_t *rounds_per_seed;  /* optional host (or device, if device_buffers) [n_seeds] out */
} labs_opts;

/* Aggregate statistics of one call (host struct, optional). */
typedef struct labs_stats {
  uint64_t evals;            /* neighbour evaluations over all seeds */
  int32_t rounds;            /* largest number of rounds any seed ran */
  int32_t launches;          /* kernels this call launched */
  int32_t walk_launches;     /* of which walk kernels */
  int32_t reserved0;
  double walk_kernel_ms;     /* sum of the walk kernels' durations (CUDA events) */
  double device_ms;          /* first to last kernel of the call (CUDA events) */
  uint64_t plane_steps;      /* sum over walk steps of the digit planes the scan used
                                (evals / D steps in all; see the design notes) */
} labs_stats;

void labs_opts_init(labs_opts *o);

/* Eq. 1 energy E of one +-1 sequence of length L (1 <= L <= 65536, any L,
 * not only skew-symmetric).  seq is a host pointer.  Returns E >= 0, or a
 * negative labs_status (LABS_EINVAL for a bad pointer, L, or a value other
 * than +1/-1; LABS_ECUDA on a device error). */
int64_t labs_energy(const int8_t *seq, int32_t L);

/* Eq. 1 energies of n sequences stored back to back (seqs[n*L], device
 * pointer) into E_out[n] (device pointer), stream-ordered on `stream`.
 * Returns LABS_EINVAL for bad sizes; a value other than +-1 is reported by
 * a LABS_EINVAL return after the stream is synchronised when check != 0. */
labs_status labs_energy_batch(const int8_t *seqs, int32_t n, int32_t L, int64_t *E_out, void *stream,
                              int32_t check);

/* Table 1's sequence code (Section 4.2, the text under Table 1): the free
 * half s_1..s_D of a skew-symmetric sequence (D = (L+1)/2) as D binary digits,
 * s_1 the most significant, +1 -> 0 and -1 -> 1, written in hexadecimal.  The
 * other half follows from Eq. 2.  Host-only format helpers: no GPU is used.
 *   labs_from_hex: hex = NUL-terminated hex digits (an optional "0x" prefix,
 *     either case, any leading zeros) -> seq_out[L] (host, caller-owned, +-1).
 *     LABS_EINVAL for a NULL pointer, an L that is not odd in
 *     LABS_L_MIN..LABS_L_MAX, a character that is not a hex digit, an empty
 *     code or a value of more than D binary digits.
 *   labs_to_hex: seq[L] (host, +-1, skew-symmetric) -> out[out_len] (host,
 *     caller-owned): ceil(D/4) upper-case hex digits, leading zeros kept (the
 *     form Table 1 prints), then a NUL.  LABS_EINVAL for a NULL pointer, a bad
 *     L, a value other than +-1, a sequence that breaks Eq. 2, or
 *     out_len < ceil(D/4) + 1. */
labs_status labs_from_hex(const char *hex, int32_t L, int8_t *seq_out);
labs_status labs_to_hex(const int8_t *seq, int32_t L, char *out, size_t out_len);

/* The whole solver (Algorithm 1 around Algorithm 2) for n_seeds independent
 * problems of the same L: rounds of walks_per_seed walks of walk_len steps,
 * until step_budget neighbour evaluations (per seed) or opts->target_E.
 *   seeds[n_seeds]       problem seeds;
 *   best_seq[n_seeds*L]  out: best sequence found for each seed (+-1);
 *   best_E[n_seeds]      out: its energy (Eq. 1);
 *   opts                 NULL = defaults; see labs_opts;
 *   stats                NULL or out.
 * Limits: 1 <= n_seeds, 1 <= walks_per_seed, n_seeds*walks_per_seed <= 2^31,
 * 1 <= walk_len <= 2^26, step_budget >= 1.  Ties between equal energies go to
 * the earliest round, then the lowest walk index.  Returns LABS_OK,
 * LABS_EINVAL, LABS_ENOMEM, LABS_ECUDA, LABS_ECHECK or LABS_EOVERFLOW. */
labs_status labs_walks(int32_t L, const uint64_t *seeds, int32_t n_seeds, int32_t walks_per_seed,
                       int32_t walk_len, uint64_t step_budget, int8_t *best_seq, int64_t *best_E,
                       const labs_opts *opts, labs_stats *stats);

/* Device bytes labs_walks needs to run all walks of a round at once (a
 * smaller opts->workspace makes it run each round in several launches; the
 * minimum is what one warp of walks needs).  0 for arguments labs_walks
 * rejects; SIZE_MAX if the size does not fit in a size_t. */
size_t labs_walks_workspace_size(int32_t L, int32_t n_seeds, int32_t walks_per_seed, int32_t walk_len);

/* One round (Eq. 4) of walks 0..n_walks-1 of the problem `seed`, with
 * per-walk results: the building block of labs_walks, exposed for checking
 * and tracing.  Host pointers; any output may be NULL.
 *   walk_best_E[n_walks], walk_best_seq[n_walks*L], walk_moves[n_walks],
 *   walk_stuck[n_walks], walk_best_step[n_walks];
 *   trace_flips[trace_count*walk_len]: the flip index chosen at every step
 *     of walks trace_begin..trace_begin+trace_count-1 (unused tail = -1);
 *   visited_keys[visited_cap*((D+63)/64)]: if not NULL, the free-bit keys of
 *     every pivot of walk `visited_walk` (bit j = 1 <-> s_{j+1} = -1), one
 *     per entry in table order, and *visited_count = how many;
 *   kernel: as labs_opts.kernel.
 * Returns like labs_walks. */
labs_status labs_saw_round(int32_t L, uint64_t seed, uint32_t round, int32_t n_walks, int32_t walk_len,
                           int32_t recheck_every, int64_t *walk_best_E, int8_t *walk_best_seq,
                           int32_t *walk_moves, int32_t *walk_stuck, int32_t *walk_best_step,
                           int32_t *trace_flips, int32_t trace_begin, int32_t trace_count,
                           int32_t visited_walk, uint64_t *visited_keys, int32_t visited_cap,
                           int32_t *visited_count, int32_t kernel);

/* ---------------------------------------------------------------- batches
 * Many independent problems of uneven L solved together (Eq. 4 rounds of
 * Algorithm 2 walks for several instances at once): a persistent kernel per
 * lag-word class W = ceil(((L-1)/2)/32) whose warps take tasks of 32 walks of
 * one round of one problem from a device counter, longest tasks first, and an
 * in-order per-problem finalize (Algorithm 1's best update and stop rule).
 * Each problem's result is exactly what labs_walks gives for it alone with
 * the same (L, seed, walks, walk_len, step_budget, target_E). */
typedef struct labs_problem {
  int32_t L;            /* odd, LABS_L_MIN..LABS_L_MAX */
  int32_t walks;        /* walks per round, 1..2^24 */
  int32_t walk_len;     /* steps per walk, 1..2^26 */
  int32_t reserved;     /* 0 */
  uint64_t seed;
  uint64_t step_budget; /* neighbour evaluations, >= 1 */
  int64_t target_E;     /* stop at the first round whose best E <= target_E; < 0 = none */
} labs_problem;

typedef struct labs_batch_opts {
  void *stream;              /* cudaStream_t; NULL = the batch creates its own stream */
  int32_t use_graph;         /* 1: when no problem has a target, the first launch sequence is
                                captured as a CUDA graph on the first run and replayed after */
  int32_t autotune;          /* 1: pick per class, by timing candidates on a sample of its first
                                launch (cached per process): one walk per lane with 64, 128 or
                                256 walks per CTA, 1.5 or 3 table slots per pivot and the scan's
                                flip loop unrolled once or twice, or one walk per warp or per
                                CTA of 128 threads (both offered while every problem has <= 4096
                                walks) */
  int32_t block_threads;     /* walks per CTA (32..256, multiple of 32) in lane mode, threads per
                                CTA in warp mode (CTA mode: always 128); 0 = 128 or autotuned */
  int32_t table_factor_x10;  /* visited-table slots per pivot x 10 (>= 12); 0 = 30 or autotuned */
  int32_t rounds_per_launch; /* rounds a problem with a target gets per launch; 0 = 4 */
  int32_t walk_mode;         /* 0: one walk per lane, or what autotune picks; 1: one walk per lane;
                                2: one walk per warp in every class; 3: one walk per CTA of 128
                                threads in every class (2 and 3: every problem <= 4096 walks,
                                else LABS_EINVAL); all give the same results */
} labs_batch_opts;

typedef struct labs_batch labs_batch; /* opaque, owns its device memory */

/* Validate the problems and allocate the batch (visited-table pools sized
 * for the device's resident lanes of each class).  problems[n] is copied.
 * Returns LABS_EINVAL for a bad problem or option, LABS_ENOMEM, LABS_ECUDA. */
labs_status labs_batch_create(const labs_problem *problems, int32_t n, const labs_batch_opts *opts,
                              labs_batch **out);
/* Solve every problem from scratch (one run = the whole solve); blocks until
 * done.  stats may be NULL. */
labs_status labs_batch_run(labs_batch *b, labs_stats *stats);
/* Result of problem i of the last run (host pointers, any may be NULL):
 * best_seq[L], best_E, evaluations, rounds.  LABS_PENDING before a run. */
labs_status labs_batch_result(const labs_batch *b, int32_t i, int8_t *best_seq, int64_t *best_E, uint64_t *evals,
                              int32_t *rounds);
/* Work accounting of problem i of the last run: the digit planes its
 * neighbourhood scans used, summed over the walk steps of its rounds. */
labs_status labs_batch_plane_steps(const labs_batch *b, int32_t i, uint64_t *plane_steps);
/* Launch shape chosen for class W (any output may be NULL): threads per CTA,
 * table factor x 10, walks resident at once, the walk's unit (0: one walk per
 * lane, 1: one walk per warp, the lanes splitting each walk's flips, 2: one
 * walk per CTA of 128 threads, its threads splitting them), and how many times
 * the scan's flip loop is unrolled (1 or 2). */
labs_status labs_batch_shape(const labs_batch *b, int32_t W, int32_t *block_threads, int32_t *table_factor_x10,
                             int32_t *resident_walks, int32_t *warp_per_walk, int32_t *unroll);
labs_status labs_batch_destroy(labs_batch *b);

/* ---------------------------------------------------------------- serving
 * A server takes solve requests (one labs_problem each) at any time and runs
 * them with continuous batching: a scheduler thread admits queued requests in
 * arrival order while a slot is free and a launch over every admitted request
 * fits half of the device arena, and keeps two launches of the persistent
 * batch kernels in flight (the next queued while one runs), each giving every
 * admitted request its next rounds.  The kernels finalize each request's
 * rounds in order as they complete and skip the rounds issued past its stop.
 * After each launch the scheduler hands back finished requests and admits new
 * ones.  A request's result is exactly what labs_walks gives for it alone.
 * Thread-safe: any host thread may submit, poll or wait; destroy must not
 * overlap other calls on the same server. */
typedef struct labs_serve_cfg {
  void *stream;              /* cudaStream_t whose queued work the server's first launch follows
                                (NULL = the legacy default stream); the server runs on streams
                                of its own */
  size_t mem_bytes;          /* device arena, allocated at create, for the visited tables and
                                task lists of the launches (two in flight, each in one half);
                                a request is admitted only while one launch over every
                                admitted request fits in half of it (default 8 GiB) */
  int32_t max_active;        /* requests admitted at once (slots), default 64 */
  int32_t max_L;             /* largest L accepted (sizes the table pools), default 301 */
  int32_t max_walks;         /* largest walks per round accepted, default 2048 */
  int32_t max_walk_len;      /* largest walk length accepted (<= 2^26), 0 = 8 * (max_L + 1) / 2 */
  int32_t rounds_per_launch; /* rounds each admitted request gets per launch, default 4 (two
                                launches are in flight: the next is queued while one runs); a
                                launch that would leave SMs idle gives requests further rounds,
                                up to 6 x rounds_per_launch in flight per request */
  int32_t block_threads;     /* threads per CTA of the batch kernels, default 128 */
  int32_t walk_mode;         /* 0: per launch and class, one walk per lane or per warp, whichever
                                keeps the GPU faster busy with the launch's tasks (rates measured
                                at create); 1: always one walk per lane; 2: always one walk per
                                warp (max_walks <= 4096, else LABS_EINVAL); same results */
} labs_serve_cfg;

typedef struct labs_result {
  int32_t status;            /* LABS_OK, or why the request ended without a result
                                (LABS_ESHUTDOWN, LABS_ECUDA, ...) */
  int32_t L;
  int64_t best_E;
  double F;                  /* L^2 / (2 best_E) */
  uint64_t evals;            /* neighbour evaluations spent */
  int32_t rounds;
  int32_t reached_target;    /* 1 if best_E <= the request's target */
  uint64_t t_submit_ns, t_admit_ns, t_done_ns; /* steady clock of the server's host */
  double p_optimal;          /* Eq. 7 for the request's evaluations: the predictive
                                model's probability that best_E is optimal
                                (labs_model_p_optimal of labs_model_nses_of_evals) */
  uint64_t plane_steps;      /* digit planes the neighbourhood scans used, summed over the
                                walk steps of the request's rounds (work accounting) */
} labs_result;

typedef struct labs_serve_stats {
  uint64_t submitted, completed, pending, active;
  uint64_t evals;            /* neighbour evaluations done so far */
  uint64_t launches, walk_launches;
  double busy_ms;            /* device time of the launches (CUDA events) */
  uint64_t mem_used;         /* arena bytes a launch over the admitted requests needs */
  int32_t status;            /* LABS_OK, or the error that stopped the server */
  int32_t reserved;
  uint64_t evals_run;        /* neighbour evaluations the device ran, including rounds run
                                speculatively past a request's stop (evals counts only the
                                rounds up to each stop) */
  uint64_t mem_peak;         /* largest share of the arena one launch used (<= mem_bytes / 2) */
  uint64_t fixed_bytes;      /* device bytes of the per-slot state, outside the arena */
  uint64_t lane_launches;          /* class kernels launched with one walk per lane, */
  uint64_t lane_unrolled_launches; /* the same with the scan's flip loop unrolled twice, */
  uint64_t warp_launches;          /* and with one walk per warp */
} labs_serve_stats;

typedef struct labs_server labs_server; /* opaque */

/* Defaults: mem_bytes 8 GiB, max_active 64, max_L 301, max_walks 2048,
 * max_walk_len 8 * (max_L + 1) / 2, rounds_per_launch 4, block_threads 128. */
void labs_serve_cfg_init(labs_serve_cfg *cfg);
/* Allocate the server (its per-slot state and round records, and the arena
 * of mem_bytes) and start its scheduler thread on the current device. */
labs_status labs_serve_create(const labs_serve_cfg *cfg, labs_server **out);
/* Queue a request; never blocks on the GPU.  LABS_EINVAL for a bad problem,
 * LABS_ENOMEM if it can never be admitted (L, walks or walk length above the
 * server's limits, or a launch over it alone would not fit half of mem_bytes), LABS_ESHUTDOWN while
 * destroying, or the error that stopped the server. */
labs_status labs_serve_submit(labs_server *s, const labs_problem *req, uint64_t *ticket);
/* LABS_PENDING while the request runs; otherwise fills *out (and best_seq[L]
 * if not NULL), forgets the ticket and returns the request's status.
 * LABS_ENOTFOUND for an unknown or already consumed ticket. */
labs_status labs_serve_poll(labs_server *s, uint64_t ticket, labs_result *out, int8_t *best_seq);
/* Like poll, but waits up to timeout_ms for the request to finish
 * (LABS_ETIMEOUT if it has not). */
labs_status labs_serve_wait(labs_server *s, uint64_t ticket, int64_t timeout_ms, labs_result *out,
                            int8_t *best_seq);
labs_status labs_serve_get_stats(labs_server *s, labs_serve_stats *out);
/* Stop the scheduler after its current launch; requests not finished by then
 * end with LABS_ESHUTDOWN.  Frees the server. */
labs_status labs_serve_destroy(labs_server *s);

/* Size of the fixed device scratch used by labs_saw_round_noalloc. */
#define LABS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* labs_saw_round_noalloc -- the same round as labs_saw_round (walks
 * 0..n_walks-1 of the problem `seed` in round `round`), for callers that
 * cannot allocate device memory: code whose device memory belongs to another
 * allocator that must not be bypassed (a framework or serving process that
 * reserves the GPU up front), processes under a hard device-memory quota, or
 * code that must not allocate on its call path.  The paper has no
 * counterpart; this is a deployment variant of its walk round.
 *
 * It calls no allocator.  Its scratch (visited tables, per-walk state,
 * counters) is one static device array of LABS_NOALLOC_SCRATCH_BYTES that
 * every process loading this library holds on every GPU it uses until exit.
 * Every output is a caller-owned device pointer to memory of the current
 * device with at least the elements stated (the library cannot check this:
 * a smaller or host buffer is written out of bounds):
 *   walk_best_E[n_walks]      int64, device out: each walk's best energy;
 *   walk_best_seq[n_walks*L]  int8, device out: each walk's best sequence (+-1);
 *   walk_moves, walk_stuck    int32 [n_walks] device out, or NULL;
 *   stream                    cudaStream_t or NULL; the call synchronises it
 *                             before returning.
 * The first call on a device looks up the scratch's device address (with
 * that device current); make that first call before any stream capture.
 * All calls in a process share the one scratch array, which keeps the last
 * call's contents (the call clears what must start at zero): calls that can
 * overlap on the GPU (other threads, other streams) race and must be
 * serialised by the caller.
 * Returns LABS_OK, LABS_EINVAL (bad L, sizes or NULL outputs), LABS_ENOMEM
 * if the round's scratch (about n_walks * (slots * 8 * ceil((D+1)/64) + 52)
 * bytes, slots = the power of two >= 3 * (walk_len + 1), at least 64)
 * exceeds LABS_NOALLOC_SCRATCH_BYTES, or LABS_ECUDA. */
labs_status labs_saw_round_noalloc(int32_t L, uint64_t seed, uint32_t round, int32_t n_walks, int32_t walk_len,
                                   int64_t *walk_best_E, int8_t *walk_best_seq, int32_t *walk_moves,
                                   int32_t *walk_stuck, void *stream);

/* ---------------------------------------------------------------------------
 * The full search space: all 2^L binary sequences of length L, any parity,
 * LABS_FULL_L_MIN <= L <= LABS_FULL_L_MAX.  The paper restricts its solver to
 * the skew-symmetric sequences and leaves the full space to future work
 * (Section 5); these functions run the same contiguous self-avoiding walks
 * (Eq. 3, Algorithm 2) and round loop (Algorithm 1) over it: a flip negates
 * one position, every step evaluates all L flips (so one step is L neighbour
 * evaluations), the visited sets hold whole sequences, and the first pivot
 * takes its L values from the Philox stream layout of the skew functions.
 * Arguments, outputs, ownership and status codes are those of the skew
 * functions above (labs_opts.kernel: 0 or 1; the incremental variant is
 * skew-only).  LABS_EINVAL for an L outside the range.
 * ------------------------------------------------------------------------- */
labs_status labs_walks_full(int32_t L, const uint64_t *seeds, int32_t n_seeds, int32_t walks_per_seed,
                            int32_t walk_len, uint64_t step_budget, int8_t *best_seq, int64_t *best_E,
                            const labs_opts *opts, labs_stats *stats);
size_t labs_walks_full_workspace_size(int32_t L, int32_t n_seeds, int32_t walks_per_seed, int32_t walk_len);
labs_status labs_saw_round_full(int32_t L, uint64_t seed, uint32_t round, int32_t n_walks, int32_t walk_len,
                                int32_t recheck_every, int64_t *walk_best_E, int8_t *walk_best_seq,
                                int32_t *walk_moves, int32_t *walk_stuck, int32_t *walk_best_step,
                                int32_t *trace_flips, int32_t trace_begin, int32_t trace_count,
                                int32_t visited_walk, uint64_t *visited_keys, int32_t visited_cap,
                                int32_t *visited_count);

/* ---------------------------------------------------------------------------
 * Predictive model of the paper (Section 4.1, Eq. 6, Eq. 7): the evaluations
 * a run needs to reach an optimal skew-symmetric sequence are exponentially
 * distributed with rate lambda(L).  Host arithmetic in double precision; no
 * GPU is involved.  Invalid arguments give NaN (or 0 for the budget).
 * ------------------------------------------------------------------------- */

/* lambda(L) = 0.006753 * 0.8617^L, the authors' trend fitted on the odd
 * L = 71..119 with known optima (Section 4.1); used beyond that range, as the
 * paper does, as an extrapolation.  NaN unless L is odd in LABS_L_MIN..LABS_L_MAX. */
double labs_model_lambda(int32_t L);
/* Eq. 6: evaluations per run (the paper's count) such that N independent runs
 * reach an optimum with probability P: ln(1 - P) / (-lambda(L) N).
 * NaN unless 0 <= P < 1 and N >= 1. */
double labs_model_nses_limit(int32_t L, double P, int32_t N);
/* Eq. 7: probability that an optimum has been reached after nses evaluations
 * (the paper's count) in total, all runs taken as one: 1 - exp(-lambda(L) nses).
 * NaN unless nses >= 0. */
double labs_model_p_optimal(int32_t L, double nses);
/* The paper's evaluation count for `evals` of this library's: the paper adds
 * D - 1 per walk step (the previous pivot is never re-evaluated), this library
 * counts all D flips of a step, so nses = evals (D - 1) / D. */
double labs_model_nses_of_evals(int32_t L, uint64_t evals);
/* The step budget (this library's evaluations, for labs_problem.step_budget or
 * labs_walks) at which Eq. 7 reaches P: ceil(nses_limit(L, P, 1) D / (D - 1)),
 * saturating at UINT64_MAX; 0 for invalid arguments. */
uint64_t labs_model_budget(int32_t L, double P);

/* Human-readable name of a status code (static string). */
const char *labs_status_str(labs_status s);

#ifdef __cplusplus
}
#endif

#endif /* LABS_H_ */
