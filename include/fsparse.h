/*
 * fsparse.h -- GB300-native Matlab-compatible sparse assembly
 *              S = sparse(i, j, s, m, n, nzmax)
 *
 * Method: S. Engblom and D. Lukarski, "Fast Matlab compatible sparse assembly
 * on multicore computers", arXiv:1406.1066.  Section numbers below refer to it.
 *
 * What the library computes (§1, §2.1, §2.2):
 *   Input  (§2.2, input listing): unit-offset int32 row indices ii[len],
 *          column indices jj[len], double values sr[len], dimensions m, n.
 *   Output (§2.1, CCS arrays under Eq. (2.1)):
 *          jcS[n+1]  column pointer, jcS[0] = 0, jcS[n] = nnz;
 *          irS[nnz]  zero-offset rows, strictly ascending inside a column;
 *          prS[nnz]  values; repeated (i, j) pairs are summed.
 *   Intermediate (§2.2, Eqs. (2.2)-(2.3), "inverse rank"):
 *          irank[len], irank[k] = CCS slot of triplet k,
 *          irS[irank[k]] = ii[k] - 1, nnz = 1 + max irank.
 *   Summation order (App. A post-processing, serial insert): every slot is
 *          the fold (((+0.0 + sr[k0]) + sr[k1]) + ...) over its triplets in
 *          ascending k.  Results are therefore deterministic to the bit and
 *          independent of launch shape; a slot whose only inputs are -0.0
 *          holds +0.0.
 *   Explicit zeros: the pattern is defined by the indices alone (Eq. (2.2));
 *          zero values and sums that cancel keep their slot.
 *
 * Conventions for every entry point:
 *   * Array pointers are DEVICE pointers (cudaMalloc, cudaMallocAsync or a
 *     framework allocator) unless a parameter name starts with h_.  The
 *     caller owns them; the library never frees them.
 *   * `stream` is a cudaStream_t passed as void*; 0 is the legacy default
 *     stream.  All device work is enqueued on it.
 *   * Sizes: the paper's indices are `int` (§2.2 listings); this library
 *     accepts len and nzmax up to 2^30 - 1 (its scan words keep two flag
 *     bits); larger -> FSPARSE_ERR_SIZE.
 *   * Errors never abort, trap or assert on the device.  Device-side
 *     findings (bad index, bounded wait expired) are written to a status
 *     word that the host reads at the final synchronisation of the
 *     symbolic phase.  On error no plan is returned (*plan_out = NULL)
 *     unless stated otherwise, and output arrays hold unspecified values.
 *   * The calls that synchronise their stream poll it (cudaStreamQuery)
 *     for up to 10 ms before blocking in cudaStreamSynchronize, so that
 *     they return within microseconds of the GPU finishing; the polling
 *     thread stays busy meanwhile.
 *   * Entry points are thread-safe with respect to distinct plans.  Calls
 *     on one plan that overlap on the GPU (different streams, no ordering)
 *     are the caller's responsibility, like any other device buffer.
 */
#ifndef FSPARSE_H
#define FSPARSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fsparse_status {
    FSPARSE_OK = 0,
    FSPARSE_ERR_ARG = 1,     /* NULL pointer, negative size/dimension, bad option  */
    FSPARSE_ERR_INDEX = 2,   /* some index < 1, or > an explicit m / n (App. A)     */
    FSPARSE_ERR_NZMAX = 3,   /* 0 < nzmax < nnz, or an output capacity below nnz    */
    FSPARSE_ERR_SIZE = 4,    /* len, nzmax or a batch total beyond 2^30 - 1         */
    FSPARSE_ERR_NOMEM = 5,   /* device allocation failed                           */
    FSPARSE_ERR_CUDA = 6,    /* a CUDA runtime call failed (see last error string) */
    FSPARSE_ERR_TIMEOUT = 7, /* a bounded device-side wait expired (no hang)       */
    FSPARSE_ERR_INTERNAL = 8 /* a kernel's own index check failed (access skipped) */
} fsparse_status;

/* Opaque, library-owned symbolic result (the "quasi assembly" state of §2.1:
   the information kept between repeated assemblies of one pattern). */
typedef struct fsparse_plan_s *fsparse_plan;
/* Opaque, library-owned concatenation of many plans for batched numerics. */
typedef struct fsparse_batch_s *fsparse_batch;

/* ------------------------------------------------------------------------
 * Symbolic assembly (§2.2-§2.3: the intermediate format irank + jcS, plus
 * irS, which Eq. (2.2) fixes from irank and ii).
 *
 *   ii, jj   device int32[len], unit-offset.  Read only.  May be NULL when
 *            len == 0.
 *   m, n     dimensions; 0 means implicit = the largest index (§2.2).
 *   nzmax    0: capacity = nnz.  nzmax >= nnz: irS/prS capacity is nzmax,
 *            slots [nnz, nzmax) hold irS = 0 / prS = +0.0 and jcS is
 *            unaffected.  0 < nzmax < nnz: FSPARSE_ERR_NZMAX.  (The paper
 *            names nzmax only in the call of §1; this is the reading used.)
 *   plan_out receives a new plan on success.
 *
 * Synchronises `stream` to read nnz and the device status word; the column
 * bucket path also reads its largest bucket once before sorting, and implicit
 * dimensions add one read of the largest indices.  Allocates the plan's
 * device arrays stream-ordered on `stream`.
 * ---------------------------------------------------------------------- */
fsparse_status fsparse_symbolic(const int32_t *ii, const int32_t *jj, int64_t len,
                                int32_t m, int32_t n, int64_t nzmax,
                                void *stream, fsparse_plan *plan_out);

/* Dimensions and sizes of a plan.  Any output pointer may be NULL.
   `cap` is the irS/prS capacity (nnz, or nzmax when larger).  Host only. */
fsparse_status fsparse_plan_info(fsparse_plan plan, int32_t *m, int32_t *n, int64_t *len,
                                 int64_t *nnz, int64_t *cap);

/* Plan-owned device arrays, valid until fsparse_plan_destroy; read only for
   the caller.  irank int32[len] (Eq. (2.2)), jcS int32[n+1], irS int32[cap].
   Any output pointer may be NULL.  irank is derived from the plan's sorted
   order the first time it is requested: a non-NULL irank argument on the
   first call launches one kernel on the legacy default stream and waits for
   it (later calls return at once). */
fsparse_status fsparse_plan_arrays(fsparse_plan plan, const int32_t **irank,
                                   const int32_t **jcS, const int32_t **irS);

/* Checkpoint and resume of the reusable symbolic state (re-assembly with the
   same pattern after a restart).  fsparse_plan_export copies the plan into a
   host buffer: a header (sizes, configuration) followed by perm, the numeric
   chunk slot bases, jcS and irS; irank is not stored (it is derived again on
   first request).  With host_buf == NULL it only reports the size in
   *bytes_out.  Synchronous (blocking copies).  fsparse_plan_import checks
   the header and every size against `bytes` before touching the device
   (FSPARSE_ERR_ARG on any mismatch), then builds a new plan on the current
   device, copying on `stream` and synchronising it before returning.  An
   imported plan behaves exactly like the exported one.  The paper has no
   counterpart (it keeps its state in memory between calls, §2). */
fsparse_status fsparse_plan_export(fsparse_plan plan, void *host_buf, int64_t capacity,
                                   int64_t *bytes_out);
fsparse_status fsparse_plan_import(const void *host_buf, int64_t bytes, void *stream,
                                   fsparse_plan *plan_out);

/* Delayed assembly (§2 names input that is not all available at the first
   call as an extension of the method): a NEW plan for the concatenation of
   the plan's triplets and (ii, jj), device int32[len] unit-offset, whose
   triplet numbers continue at the plan's len.  The result equals
   fsparse_symbolic on the concatenated arrays with the plan's m and n: the
   appended indices must lie within them (FSPARSE_ERR_INDEX otherwise, no
   plan).  Values for fsparse_numeric on the new plan are the old values
   followed by the new ones.  The new plan's capacity is its nnz (the old
   plan's nzmax tail is not carried over).  The old plan is not modified and
   stays valid; the caller destroys both.  Synchronises `stream`. */
fsparse_status fsparse_plan_append(fsparse_plan plan, const int32_t *ii, const int32_t *jj,
                                   int64_t len, void *stream, fsparse_plan *plan_out);

/* Release a plan (NULL is a no-op).  Neither the host nor the device as a
   whole waits: the plan's arrays go back to the stream-ordered pool, on a
   stream of the library's, once (1) every fsparse_numeric and
   fsparse_numeric_adjoint launch on the plan has finished (the library
   records an event per stream after each of them; launches captured into a
   CUDA graph are not recorded) and (2) the work queued so far on the legacy
   default stream -- and with it on every blocking stream -- has finished.
   Reads of the plan's arrays that the caller queued itself on non-blocking
   streams, and replays of captured graphs, must be finished or ordered
   before this call, as for any device buffer.  fsparse_plan_release does
   the same and also orders the release after the work queued so far on
   `stream`. */
fsparse_status fsparse_plan_destroy(fsparse_plan plan);
fsparse_status fsparse_plan_release(fsparse_plan plan, void *stream);

/* ------------------------------------------------------------------------
 * Numeric assembly (Eq. (2.3); App. A post-processing): prS[slot] is the
 * ascending-k fold from +0.0 of sr[k] over the triplets of that slot.
 *
 *   sr   device double[len] in the triplet order of the symbolic call.
 *   prS  device double[cap] (cap from fsparse_plan_info); fully written,
 *        including the zero tail [nnz, cap).
 *
 * No synchronisation, no allocation, no validation of values: safe to call
 * repeatedly on new values of one pattern (re-assembly in time-dependent
 * nonlinear PDE solvers, §1) and to record into a CUDA graph.
 * ---------------------------------------------------------------------- */
fsparse_status fsparse_numeric(fsparse_plan plan, const double *sr, double *prS, void *stream);

/* Adjoint (transpose) of the numeric map, which is linear in sr (Eq. (2.3)):
   ds[k] = dprS[irank[k]] for k < len.  dprS device double[>= nnz], ds device
   double[len].  Exact (a gather, no rounding).  No sync, no allocation; the
   first adjoint call on a plan whose irank was never requested also
   launches the kernel that derives irank, on `stream`. */
fsparse_status fsparse_numeric_adjoint(fsparse_plan plan, const double *dprS, double *ds,
                                       void *stream);

/* ------------------------------------------------------------------------
 * Full assembly: symbolic + numeric in one call, S = sparse(i,j,s,m,n,nzmax)
 * of §1.  prS is caller-owned with `prS_capacity` doubles.  The CCS arrays
 * jcS and irS are the returned plan's (fsparse_plan_arrays).
 *
 * When prS_capacity >= max(len, nzmax) the values are folded inside the
 * symbolic pass; otherwise the numeric pass runs after nnz is known, and a
 * capacity below the plan's cap returns FSPARSE_ERR_NZMAX WITH the plan
 * (*plan_out set), so the caller can allocate and call fsparse_numeric.
 * plan_out must not be NULL.  Synchronises `stream` as fsparse_symbolic does.
 * ---------------------------------------------------------------------- */
fsparse_status fsparse_assemble(const int32_t *ii, const int32_t *jj, const double *sr,
                                int64_t len, int32_t m, int32_t n, int64_t nzmax,
                                double *prS, int64_t prS_capacity, void *stream,
                                fsparse_plan *plan_out);

/* ------------------------------------------------------------------------
 * Matlab-style double index arrays (App. A pre-processing of the index
 * input): ii and jj are device double[len] holding unit-offset indices, as
 * Matlab passes them.  Each value must be at least 1.0 and equal to its
 * ceiling (an integer; NaN fails); this library also rejects values above
 * 2^31 - 1, which the paper's int cannot hold.  A rejected value gives
 * FSPARSE_ERR_INDEX and no plan, exactly as an out-of-range int index does.
 * Otherwise the calls behave as fsparse_symbolic / fsparse_assemble on the
 * converted indices (same arguments, results, ownership and synchronisation);
 * the conversion uses 8*len bytes of temporary device memory from the same
 * stream-ordered pool, handed back to the pool (in stream order) before the
 * call returns.
 * ---------------------------------------------------------------------- */
fsparse_status fsparse_symbolic_f64(const double *ii, const double *jj, int64_t len, int32_t m,
                                    int32_t n, int64_t nzmax, void *stream, fsparse_plan *plan_out);

fsparse_status fsparse_assemble_f64(const double *ii, const double *jj, const double *sr,
                                    int64_t len, int32_t m, int32_t n, int64_t nzmax,
                                    double *prS, int64_t prS_capacity, void *stream,
                                    fsparse_plan *plan_out);

/* ------------------------------------------------------------------------
 * Batched numeric re-assembly of many independent patterns (many small
 * assemblies per time step).  The batch concatenates `count` plans: triplet
 * k of plan b is element h_len_off[b] + k of the concatenated sr, and slot
 * p < nnz_b of plan b is element h_nnz_off[b] + p of the concatenated prS,
 * where the offsets are exclusive prefix sums of each plan's len and nnz
 * (read them with fsparse_batch_info; zero tails from nzmax are not part of
 * a batch).  The total len must stay below 2^30.  The plans may be destroyed
 * after the batch is created.  Synchronises `stream` once.
 * ---------------------------------------------------------------------- */
fsparse_status fsparse_batch_create(int32_t count, const fsparse_plan *h_plans, void *stream,
                                    fsparse_batch *batch_out);

/* ------------------------------------------------------------------------
 * Batched symbolic assembly: `count` independent instances in ONE symbolic
 * pass (re-assembly of many patterns per time step, §1; the reusable
 * "quasi assembly" state of §2.1 for all of them at once).
 *
 *   ii, jj     device int32[h_len_off[count]]: the instances' unit-offset
 *              triplets, concatenated; instance b owns positions
 *              [h_len_off[b], h_len_off[b+1]).  Read only.
 *   h_len_off  HOST int64[count+1], h_len_off[0] = 0, non-decreasing.
 *   h_m, h_n   HOST int32[count]: each instance's dimensions; 0 means
 *              implicit = that instance's largest index (§2.2; costs one
 *              extra synchronisation for the whole batch).
 *   batch_out  receives a new batch.
 *
 * Every instance is assembled exactly as fsparse_symbolic would assemble it
 * alone (nzmax 0): the batch is the single problem [S_0 S_1 ... S_{count-1}]
 * -- the instances' matrices side by side, instance b's columns shifted by
 * n_0 + ... + n_{b-1} -- so its column-compressed arrays hold every
 * instance's arrays in order.  fsparse_batch_numeric on the result equals
 * fsparse_numeric per instance, bit for bit, with instance b's values at
 * h_len_off[b] of sr_concat and its prS at h_nnz_off[b] of prS_concat
 * (fsparse_batch_info).  An index outside its own instance's m x n, or
 * below 1, returns FSPARSE_ERR_INDEX and no batch.  The total length must
 * stay below 2^30 and the instances' columns must add up to at most
 * 2^31 - 1 (FSPARSE_ERR_SIZE).  Synchronises `stream` (as fsparse_symbolic,
 * plus one read of the instances' slot offsets); allocates stream-ordered.
 * ---------------------------------------------------------------------- */
fsparse_status fsparse_batch_symbolic(int32_t count, const int32_t *ii, const int32_t *jj,
                                      const int64_t *h_len_off, const int32_t *h_m,
                                      const int32_t *h_n, void *stream, fsparse_batch *batch_out);

/* The per-instance CCS arrays of a batch made by fsparse_batch_symbolic,
   concatenated; batch-owned device arrays, valid until the batch is
   destroyed, read only for the caller.  Any pointer may be NULL.
     irank  int32[total len]: instance b's irank (its own slot numbers) at
            h_len_off[b];
     jcS    int32[sum over b of (n_b + 1)]: instance b's jcS (starting at 0)
            at n_0 + ... + n_{b-1} + b;
     irS    int32[total nnz]: instance b's irS at h_nnz_off[b];
     h_m, h_n  HOST int32[count]: the dimensions used (implicit ones resolved).
   irank is derived on the first request that asks for it (one kernel pair on
   the legacy default stream, waited for).  A batch made from plans
   (fsparse_batch_create) keeps these arrays in its plans: FSPARSE_ERR_ARG. */
fsparse_status fsparse_batch_arrays(fsparse_batch batch, const int32_t **irank, const int32_t **jcS,
                                    const int32_t **irS, int32_t *h_m, int32_t *h_n);

/* Host offsets: h_len_off and h_nnz_off receive count+1 int64 each (either
   may be NULL).  Host only. */
fsparse_status fsparse_batch_info(fsparse_batch batch, int32_t *count, int64_t *h_len_off,
                                  int64_t *h_nnz_off);

/* All instances in ONE launch (a persistent kernel over the concatenated
   triplet space); bit-identical to calling fsparse_numeric per plan.  No
   sync, no allocation: capturable in a CUDA graph. */
fsparse_status fsparse_batch_numeric(fsparse_batch batch, const double *sr_concat,
                                     double *prS_concat, void *stream);

/* Release a batch; same ordering rules as fsparse_plan_destroy /
   fsparse_plan_release (the recorded launches are fsparse_batch_numeric). */
fsparse_status fsparse_batch_destroy(fsparse_batch batch);
fsparse_status fsparse_batch_release(fsparse_batch batch, void *stream);

/* ------------------------------------------------------------------------
 * Column-sharded assembly on several GPUs (one process per GPU): the
 * routing steps.  The paper's multicore method (§3) gives every thread a
 * contiguous range of rows; across GPUs every rank owns a contiguous range
 * of COLUMNS, h_col_split[r] < j <= h_col_split[r+1] (unit-offset j), so
 * every slot -- and every column of jcS, irS and prS -- belongs to exactly
 * one rank, and the output is distributed by column blocks (§2 names a
 * distributed output as an extension of the method).  The collectives
 * themselves (an all-to-all of the routed triplets, an exclusive scan of
 * the ranks' nnz) are the caller's; the Python module
 * paper_1406_1066_gb300.shard runs them with torch.distributed.
 *
 * fsparse_shard_route: rank r's slice of the triplets (device ii, jj int32
 * [len] unit-offset, sr double[len] or NULL) is partitioned stably by
 * destination rank: the send arrays (device, [len] each) hold the triplets
 * for rank 0 first, then rank 1, ..., each group in ascending position of
 * the slice; send_j holds the column INSIDE the destination's block
 * (j - h_col_split[dest], unit offset); send_s the values (left alone when
 * sr is NULL); send_k the slice position of every routed triplet (keep it:
 * it is the route).  h_counts (host int64[nranks]) receives the group
 * sizes.  Indices are validated against m, n (> 0): a bad one gives
 * FSPARSE_ERR_INDEX.  nranks 1..256, h_col_split host int64[nranks+1] from 0
 * to n, non-decreasing.  Synchronises `stream` once.
 *
 * When the slices are taken in rank order and received in source-rank
 * order, each rank's received triplets are in global triplet order, so its
 * local fsparse_assemble sums every slot in ascending global k: the result
 * is the single-GPU assembly, bit for bit, cut into column blocks.
 *
 * fsparse_shard_unroute: out[send_k[p]] = back[p] for p < len (device int32
 * arrays): the values returned for the routed triplets (e.g. their global
 * slots) land at the slice positions they came from.
 * fsparse_shard_gather: send_s[p] = sr[send_k[p]]: new values along a kept
 * route (numeric re-assembly of a sharded pattern).  fsparse_shard_offset:
 * out[p] = in[p] + add (device int32, in place allowed): a rank's local slot
 * numbers and column pointers shifted by its slot offset, the exclusive
 * scan of the ranks' nnz.  All three: no sync, no allocation.
 * ---------------------------------------------------------------------- */
fsparse_status fsparse_shard_route(const int32_t *ii, const int32_t *jj, const double *sr, int64_t len,
                                   int32_t m, int32_t n, int32_t nranks, const int64_t *h_col_split,
                                   int32_t *send_i, int32_t *send_j, double *send_s, int32_t *send_k,
                                   int64_t *h_counts, void *stream);
fsparse_status fsparse_shard_unroute(const int32_t *back, const int32_t *send_k, int64_t len, int32_t *out,
                                     void *stream);
fsparse_status fsparse_shard_gather(const double *sr, const int32_t *send_k, int64_t len, double *send_s,
                                    void *stream);
fsparse_status fsparse_shard_offset(const int32_t *in, int64_t len, int64_t add, int32_t *out, void *stream);

/* ------------------------------------------------------------------------
 * Launch configuration and autotuning (library-specific; the paper's
 * method has no tuning knobs).
 *
 * strategy: FSPARSE_SORT_ONESWEEP = global stable LSD radix sort of the
 * packed (column,row) keys, one kernel per digit with decoupled look-back;
 * FSPARSE_SORT_BUCKET = one partition by the high column bits (a count and
 * a scatter, each run once per range of 32,768 buckets; order inside a
 * bucket is not kept), then one shared-memory pass per column bucket fused
 * with run detection, the ascending-k order inside every run, jcS and the
 * chunk slot bases.  Inside a bucket whose (column, dense row rank) key
 * space fits a 65,536-bit map the unique keys are counted in that bitmap (no
 * sort pass); other buckets take 8-bit radix passes.
 * FSPARSE_SORT_BUCKET_RADIX = the same with the radix passes in every bucket.
 * All give bit-identical results.  A bucket that outgrows shared memory, or
 * one (i,j) pair repeated more than 384 times, makes the library redo the
 * call with ONESWEEP (same results, more time).
 * ---------------------------------------------------------------------- */
typedef enum fsparse_strategy {
    FSPARSE_SORT_AUTO = 0,
    FSPARSE_SORT_ONESWEEP = 1,
    FSPARSE_SORT_BUCKET = 2,
    FSPARSE_SORT_BUCKET_RADIX = 3
} fsparse_strategy;

typedef struct fsparse_config {
    int32_t strategy;        /* fsparse_strategy                                 */
    int32_t radix_bits;      /* ONESWEEP digit width, 6..8 (9, 10: 256 threads)  */
    int32_t sweep_items;     /* ONESWEEP items per thread: 8, 12 or 16            */
    int32_t sweep_threads;   /* ONESWEEP threads per block: 256 or 512            */
    int32_t bucket_target;   /* BUCKET mean items per bucket, 1024..16384         */
    int32_t numeric_tile;    /* positions per numeric tile: 1024, 2048 or 4096    */
} fsparse_config;

/* The configuration the library would use for this problem shape (pure host
   computation; no device access).  Precedence: fsparse_set_config override,
   then the tuned table, then built-in defaults. */
fsparse_status fsparse_get_config(int64_t len, int32_t m, int32_t n, fsparse_config *out);

/* Per-phase device time of the calling thread's last symbolic, assemble or
   append call, recorded when FSPARSE_TIMING=1 is set for that call (CUDA events on
   its stream, read at its final synchronisation; a call made without it
   records nothing).  Writes up to `max` phase names
   (static strings, e.g. "bucket_count", "bucket_scatter", "bucket_emit",
   "digit_hist", "digit_passes", "emit", "jcS_scan", "numeric_fold"; an
   append adds "append_symbolic" and the "merge_*" phases) and
   durations in ms; returns the number of phases recorded (0 when none).
   Either array may be NULL.  Host only. */
int32_t fsparse_last_timings(const char **names, double *ms, int32_t max);

/* Process-wide override (NULL clears it).  Fields <= 0 keep the value that
   would otherwise apply.  Invalid values: FSPARSE_ERR_ARG.  Host only. */
fsparse_status fsparse_set_config(const fsparse_config *cfg);

/* Tune on the given device problem (the inputs are only read), timing with
   CUDA events on `stream`: first every sort configuration by the time of the
   symbolic call (`reps` timed runs each, >= 1), then the numeric tile by
   repeated folds on the winner's plan.  The result is kept for the problem's
   size class in the process-wide table and reported in *best (may be NULL).
   Allocates and synchronises freely; not for use inside graph capture. */
fsparse_status fsparse_autotune(const int32_t *ii, const int32_t *jj, const double *sr,
                                int64_t len, int32_t m, int32_t n, int32_t reps,
                                void *stream, fsparse_config *best);

/* Persist / restore the tuned table as JSON (host files). */
fsparse_status fsparse_tune_save(const char *path);
fsparse_status fsparse_tune_load(const char *path);
/* Forget every tuned entry (the override set by fsparse_set_config stays). */
fsparse_status fsparse_tune_clear(void);

/* ------------------------------------------------------------------------
 * Assembly without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that are not allowed to allocate GPU
 * memory themselves or through this library -- code running under another
 * framework's memory manager or arena, solver loops that forbid allocation
 * after start-up, plug-ins that only receive pre-allocated buffers.
 *
 * Same result as fsparse_assemble (bit for bit) for problems within the
 * limits below, written to caller-owned device buffers: irank int32[len],
 * jcS int32[n+1], irS int32[len], prS double[len] (the first *nnz_out
 * entries of irS/prS are the CCS arrays).  m and n must be given (> 0);
 * there is no nzmax and no plan.  *nnz_out is a HOST int64.
 *
 * Working memory: one static device array of FSPARSE_NOALLOC_SCRATCH_BYTES
 * inside this library, which every GPU that loads the library keeps until
 * the process exits.  The entry point calls no cudaMalloc, cudaFree or other
 * allocating routine.  Every call looks up that array's device address on the
 * current device (cudaGetSymbolAddress), so a device reset between calls is
 * harmless; the first call on each device also loads the array, and should
 * come before any stream capture.  All calls share the one array: calls that overlap on the
 * GPU (other streams or threads, without ordering) race and must not be
 * issued.  Synchronises `stream` once to read nnz.
 *
 * len > FSPARSE_NOALLOC_MAX_LEN or n > FSPARSE_NOALLOC_MAX_COLS returns
 * FSPARSE_ERR_SIZE before touching the device.
 * ---------------------------------------------------------------------- */
#define FSPARSE_NOALLOC_MAX_LEN 131072
#define FSPARSE_NOALLOC_MAX_COLS 131072
#define FSPARSE_NOALLOC_SCRATCH_BYTES (5u << 20)

fsparse_status fsparse_assemble_noalloc(const int32_t *ii, const int32_t *jj, const double *sr,
                                        int64_t len, int32_t m, int32_t n, int32_t *irank,
                                        int32_t *jcS, int32_t *irS, double *prS,
                                        int64_t *nnz_out, void *stream);

/* ------------------------------------------------------------------------
 * Diagnostics.
 * ---------------------------------------------------------------------- */
/* Human-readable text of the last error raised on the calling thread. */
const char *fsparse_last_error_string(void);
/* Static name of a status code. */
const char *fsparse_status_string(fsparse_status status);
/* Number of kernels this library has launched in this process. */
int64_t fsparse_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* FSPARSE_H */
