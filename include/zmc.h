/*
 * zmc.h -- C ABI of the GB300 multi-function direct Monte Carlo integrator.
 *
 * The method is the multi-function mode of ZMCintegral-v5.1 (arXiv
 * 2104.10073): many integrands, each with its own form, dimension and box
 * domain (Sec. "Summary of revisions": Eq. 1, Eq. 2 and the text after it),
 * integrated together by direct Monte Carlo, one estimate per integrand
 * (Sec. "Solution method"), with the estimate's spread reported beside it
 * (Fig. 1 caption).
 *
 * For integrand f on the box B = prod_i [lo_i, hi_i] with N samples:
 *     estimate = V * mean,   V = prod_i (hi_i - lo_i),  mean = (1/N) sum_s f(x_s)
 *     stderr   = V * sqrt(M2 / (N (N - 1))),            M2 = sum_s (f(x_s) - mean)^2
 * Sample s of an integrand with dimension d, key `seed` and stream `stream_id`
 * uses 23-bit fields c = s*d + i (i < d) of a Philox4x32-10 stream: field c is
 * bits 23k .. 23k+22 (k = c mod 5) of the 128-bit output, word 0 least
 * significant, of Philox4x32-10(counter = (stream_id, b mod 2^32, b div 2^32, 0),
 * key = (seed mod 2^32, seed div 2^32)), b = c div 5, and coordinate i is
 * x_i = lo_i + (hi_i - lo_i) * field * 2^-23.  The results are
 * therefore a pure function of the descriptor table: they do not depend on
 * launch configuration, on which other integrands share a launch, or on how
 * work is split between launches.
 *
 * Conventions for every entry point:
 *   - Pointers are plain host pointers unless the argument says "device".
 *     The caller owns every array it passes; the library copies what it keeps.
 *   - Every call returns a zmc_status.  On failure zmc_last_error() gives a
 *     one-line reason.  A CUDA error returns ZMC_ECUDA and leaves the context
 *     unusable (every later call on it returns ZMC_ECUDA); destroy it.
 *   - A context serialises its calls internally; different contexts are
 *     independent.
 *   - A table of descriptors holds n >= 1 rows: an empty table (n = 0) is
 *     rejected with ZMC_EINVAL by every call that integrates, plans or submits
 *     it, since there is nothing to integrate.  zmc_validate accepts it (no row
 *     is invalid); the test calls zmc_philox4x32_10 (n = 0) and
 *     zmc_eval_samples (count = 0) return ZMC_OK without computing anything.
 */
#ifndef ZMC_H
#define ZMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZMC_MAX_DIM 7
#define ZMC_NPARAM 40

/* Integrand families.  x is the point, d the dimension; parameter layout in
 * zmc_desc.p:
 *   ZMC_HARMONIC  a cos(k.x) + b sin(k.x)        (Eq. 1)   p[0]=a p[1]=b p[2+i]=k_i
 *   ZMC_ABSLIN    a |c.x|                        (Eq. 2)   p[0]=a p[1+i]=c_i
 *   ZMC_GAUSS     A exp(-|x-mu|^2 / (2 sigma^2))           p[0]=A p[1]=sigma p[2+i]=mu_i
 *   ZMC_POLY      prod_i sum_{j<=deg} c_ij x_i^j          p[5i+j]=c_ij              */
enum zmc_family {
    ZMC_HARMONIC = 0,
    ZMC_ABSLIN = 1,
    ZMC_GAUSS = 2,
    ZMC_POLY = 3,
    ZMC_USER = 4 /* a user-defined integrand: only through zmc_udf_integrate        */
};

typedef enum zmc_status {
    ZMC_OK = 0,
    ZMC_EINVAL = 1,    /* bad argument or descriptor                               */
    ZMC_ENOMEM = 2,    /* the request can never fit the device memory budget       */
    ZMC_EAGAIN = 3,    /* zmc_poll: the job is not finished yet                    */
    ZMC_ETIMEOUT = 4,  /* zmc_poll: waited wait_ms and the job is still running    */
    ZMC_ECUDA = 5,     /* a CUDA call failed; the context is poisoned              */
    ZMC_ENOTFOUND = 6, /* unknown or already collected job id                      */
    ZMC_ECLOSED = 7,   /* the context is shutting down / job was cancelled         */
    ZMC_ENOSYS = 8     /* feature not available in this build                      */
} zmc_status;

/* One integrand (464 bytes, naturally aligned, no padding beyond `deg`).
 * Valid: family in 0..3, 1 <= dim <= 7, 1 <= n_samples <= 2^62, lo_i < hi_i
 * finite, deg <= 4 (ZMC_POLY; 0 otherwise), sigma > 0 (ZMC_GAUSS), all 40
 * parameters finite, and the FP32 evaluation constants derived from them in
 * range:
 *   - ZMC_HARMONIC: |k_i (hi_i - lo_i)| / (2 pi) <= 2^20 turns per dimension and
 *     |k.lo - atan2(b, a)| / (2 pi) < 4e15 turns (the fixed-point phase), and
 *     sqrt(a^2 + b^2) times the power-of-two scale finite in FP32;
 *   - ZMC_ABSLIN: c.lo, sum |c_i| max(|lo_i|, |hi_i|) finite, and a 2^-F times
 *     the scale a normal FP32 number or 0 (F the fixed-point exponent of c.x);
 *   - ZMC_GAUSS, ZMC_POLY: every scaled constant (amplitude, 1/sigma terms,
 *     coefficients re-expanded on the unit box) finite in FP32.
 * (The scale is 2^(48 - ceil(log2 B)), B a bound of |f| on the box, clamped
 * to 2^-100 .. 2^100.)  A row outside these rules is rejected with ZMC_EINVAL
 * and a reason in zmc_last_error(); zmc_validate applies the same rules.
 * Entries of lo/hi/p beyond the family's use are ignored.                      */
typedef struct zmc_desc {
    uint32_t family;
    uint32_t dim;
    uint32_t stream_id; /* Philox counter word 0: selects the integrand's stream */
    uint32_t deg;
    uint64_t n_samples;
    uint64_t seed;      /* Philox key                                             */
    double lo[ZMC_MAX_DIM];
    double hi[ZMC_MAX_DIM];
    double p[ZMC_NPARAM];
} zmc_desc;

/* One result.  status is ZMC_OK, or ZMC_ECLOSED for a cancelled job's rows.
 * stderr_ is NaN when n == 1 (the spread of one sample is undefined).        */
typedef struct zmc_result {
    double estimate;
    double stderr_;
    uint64_t n;
    int32_t status;
    int32_t reserved;
} zmc_result;

/* Moments of f over a sample range: n samples, their mean and
 * M2 = sum (f - mean)^2 (not multiplied by the volume).  status as in zmc_result. */
typedef struct zmc_moments {
    double mean;
    double m2;
    uint64_t n;
    int32_t status;
    int32_t reserved;
} zmc_moments;

typedef struct zmc_options {
    uint64_t mem_budget_bytes;   /* device arena; 0 -> 1 GiB                          */
    void *arena;                 /* optional caller-owned DEVICE buffer of
                                    mem_budget_bytes bytes (e.g. a framework tensor),
                                    256-byte aligned; NULL -> the library allocates */
    void *stream;                /* cudaStream_t for all work; NULL -> the library
                                    creates a non-blocking stream                   */
    uint32_t max_chunks_per_iter;/* serving: chunks per persistent launch; 0 -> the
                                    chunks of 2^31 samples                          */
    uint32_t autotune;           /* flags (0: none):
                                    ZMC_TUNE_GEOMETRY: time launch geometries of each
                                    family kernel on a slice of a new plan's work (or
                                    reuse the cache); never changes results.
                                    ZMC_TUNE_CHUNK: also pick, per plan, the chunk
                                    length (quints_per_lane among 26, 52, 104, 208)
                                    and each family kernel's quint-loop unroll (1 or
                                    2), timed on a bounded subset of the table's rows
                                    and cached by the table's shape class (families,
                                    dominant dimensions, size).  Both change results
                                    within rounding only: results are bit-identical
                                    for a given choice (zmc_plan_info reports it),
                                    and unroll 1 is the untuned kernel.  Plans
                                    of sample ranges (zmc_integrate_moments) keep
                                    quints_per_lane.                                */
    int32_t device;              /* CUDA device ordinal                              */
    uint32_t quints_per_lane;    /* chunk = 160 * quints_per_lane samples (a quint
                                    is 5 consecutive samples); 0 -> 104, or 26 when
                                    serving is set.
                                    Results are bit-identical for a fixed value and
                                    agree within rounding across values.            */
    const char *tune_cache_path; /* autotune JSON cache; NULL -> no file             */
    uint32_t serving;            /* 1: start the serving thread (zmc_submit/poll)    */
    uint32_t serving_share;      /* serving: how a launch's chunks are shared.
                                    0: oldest job first (its next chunks up to the
                                    launch's budget, what is left to the next job);
                                    > 0: an equal share for every job with work
                                    left, at least this many chunks each          */
    uint32_t reserved;
    uint64_t serving_cut_backlog;/* serving, oldest first: while fewer than this
                                    many samples are left to issue over the live
                                    jobs, a launch ends with the last chunks of the
                                    first job it completes (that job's results do
                                    not wait for newer jobs' chunks; they start the
                                    next launch); with a longer backlog every launch
                                    is filled to its budget.  0 -> 2^34 (about 47 ms
                                    of sampling on one GB300); 1 -> every launch
                                    filled.  Results do not depend on it.          */
} zmc_options;

#define ZMC_TUNE_GEOMETRY 1u
#define ZMC_TUNE_CHUNK 2u

typedef struct zmc_ctx zmc_ctx;
typedef struct zmc_plan zmc_plan;

typedef struct zmc_plan_info {
    uint64_t n_fn;
    uint64_t n_chunks;     /* work items of the persistent launch                  */
    uint64_t n_samples;    /* total samples over all integrands                    */
    uint32_t grid;         /* largest persistent grid over the family kernels      */
    uint32_t block;        /* default threads per block                            */
    uint32_t quints_per_lane;
    uint32_t sms;
    uint32_t family_grid[4];   /* per family kernel (harmonic, abs-linear, Gaussian, */
    uint32_t family_block[4];  /* polynomial); block 0 = family absent             */
    int32_t tune_source[4];    /* 0 default geometry, 1 measured by the autotuner,  */
                               /* 2 taken from the autotune cache                   */
    uint32_t family_unroll[4]; /* quint-loop unroll of each family kernel (1 or 2)  */
    int32_t chunk_tune_source; /* chunk length and unroll: 0 default (quints_per_lane
                                  of the context, unroll 1), 1 measured, 2 cached   */
    uint32_t reserved;
} zmc_plan_info;

typedef struct zmc_serving_stats {
    uint64_t submitted, completed, cancelled, queued, running;
    uint64_t iterations;         /* persistent launches so far                     */
    uint64_t samples_done;
    uint64_t arena_used_bytes, arena_bytes;
    uint64_t shared_iterations;  /* launches whose work items came from >= 2 jobs   */
    uint64_t max_jobs_per_iter;  /* most jobs with work items in one launch so far  */
} zmc_serving_stats;

/* Fill *opt with defaults (1 GiB arena, own stream, device 0, no autotune). */
zmc_status zmc_default_options(zmc_options *opt);

/* Create a context on opt->device.  Allocates the arena (unless given), a
 * pinned host staging buffer and, if opt->serving, starts the scheduler thread.
 * *out is set on success and must be released with zmc_destroy. */
zmc_status zmc_create(const zmc_options *opt, zmc_ctx **out);

/* Stop the serving thread (pending jobs are cancelled), wait for the stream,
 * free everything the context owns.  NULL is accepted. */
zmc_status zmc_destroy(zmc_ctx *ctx);

/* Reason for the last failure on this thread (ctx may be NULL).  Valid until
 * the next call on this thread. */
const char *zmc_last_error(zmc_ctx *ctx);

/* Blocking batched integration of n descriptors (host arrays in and out):
 * validate and precompute on the host, copy the table to the device, run the
 * persistent FP32 sampling launch over all (integrand, chunk) work items and
 * the FP64 merge, copy the n results back. */
zmc_status zmc_integrate(zmc_ctx *ctx, const zmc_desc *desc, size_t n, zmc_result *out);

/* Same results contract computed the plain way: one FP64 direct-MC kernel
 * launch per integrand (FP64 map and evaluation, FP64 reductions), then one
 * merge launch.  The baseline the batched form is measured against. */
zmc_status zmc_integrate_plain(zmc_ctx *ctx, const zmc_desc *desc, size_t n,
                               zmc_result *out);

/* Moments of desc[i]'s integrand over samples [s_begin[i], s_end[i]) of its
 * stream (host arrays; s_begin a multiple of 5, s_begin < s_end; desc[i].n_samples
 * is ignored).  Because every sample is addressed by its Philox counter, pieces
 * of one stream combine exactly: for pieces a, b with d = mean_b - mean_a,
 *     n = n_a + n_b,  mean = mean_a + d n_b / n,  M2 = M2_a + M2_b + d^2 n_a n_b / n
 * (Chan et al.), and estimate = V mean, stderr = V sqrt(M2 / (n (n-1))) of the
 * merged moments give zmc_integrate's result for the union of the pieces (equal up
 * to FP64 rounding; chunk-aligned boundaries, multiples of 160 * quints_per_lane,
 * reproduce the same FP32 chunk sums).  This is how one stream is split over
 * GPUs or processes, checkpointed between pieces, or extended to more samples
 * later.  Blocking, like zmc_integrate. */
zmc_status zmc_integrate_moments(zmc_ctx *ctx, const zmc_desc *desc, const uint64_t *s_begin,
                                 const uint64_t *s_end, size_t n, zmc_moments *out);

/* Functional mode: one integrand form over many parameter points (the paper's
 * ZMCintegral_functional use case, Sec. "Solution method" and "Additional
 * comments": middle-dimensional integrands over a large parameter space).
 * Point q is `base` with slot slots[k] set to values[q * n_slots + k]; slot j < 40
 * is p[j], 40 + i is lo[i], 47 + i is hi[i] (ZMC_SLOT_* below).  Point q's stream
 * is base.stream_id + q if independent_streams is nonzero, else base.stream_id
 * for every point (common random numbers: all points see the same sample
 * points, so differences between points carry no noise from changing samples).
 * Results for the n_points points go to out (host).  Blocking. */
#define ZMC_SLOT_P(j) (j)
#define ZMC_SLOT_LO(i) (40 + (i))
#define ZMC_SLOT_HI(i) (47 + (i))
zmc_status zmc_integrate_functional(zmc_ctx *ctx, const zmc_desc *base, const uint32_t *slots,
                                    uint32_t n_slots, const double *values, size_t n_points,
                                    uint32_t independent_streams, zmc_result *out);

/* Serving (continuous batching).  zmc_submit copies the n descriptors into a
 * job and returns its id at once; the scheduler admits queued jobs as device
 * memory frees up, keeps their partial sums on the device, and fills each
 * persistent launch with the admitted jobs' chunks, oldest job first (or in
 * equal shares, opt->serving_share); while the backlog is short a launch ends
 * with the first job it completes (opt->serving_cut_backlog).  A job's results
 * do not depend on which jobs share its launches.  A job that alone exceeds the
 * memory budget is refused with ZMC_ENOMEM; a job may hold at most 43690
 * integrands (ZMC_EINVAL beyond).
 * Requires opt->serving = 1. */
zmc_status zmc_submit(zmc_ctx *ctx, const zmc_desc *desc, size_t n, uint64_t *job_id);

/* Collect a job.  wait_ms = 0: return ZMC_EAGAIN if it is not finished;
 * wait_ms > 0: wait up to that long, then ZMC_ETIMEOUT; wait_ms < 0: wait until
 * done.  On ZMC_OK the job's n results are written to out (n entries, in
 * submission order) and the id is released (a second poll gives ZMC_ENOTFOUND). */
zmc_status zmc_poll(zmc_ctx *ctx, uint64_t job_id, zmc_result *out, int32_t wait_ms);

/* Cancel a queued or running job; a later poll returns ZMC_ECLOSED. */
zmc_status zmc_cancel(zmc_ctx *ctx, uint64_t job_id);

/* Checkpoint a job and release it (preemption, migration, shutdown).  The job
 * stops receiving chunks at once; when the chunks already in flight have
 * finished, out[i] (n entries, host) holds the moments of every sample integrand
 * i has taken so far -- the first out[i].n samples of its stream, a multiple of
 * 160 * quints_per_lane unless the integrand is complete -- including the moments
 * it was resumed from.  A queued job is released at once with its starting
 * moments (n = 0 for a fresh job).  Samples are addressed by their Philox
 * counter (Sec. "Solution method": direct MC per integrand; the generator is
 * counter-based), so zmc_submit_resume continues each stream exactly where the
 * checkpoint stopped, on this or any other context.
 * wait_ms as in zmc_poll; after ZMC_ETIMEOUT the checkpoint stays under way and
 * a later call with the same id collects it.  A job that has already issued all
 * of its samples is not stopped: ZMC_EAGAIN, collect it with zmc_poll.  A later
 * zmc_poll of a checkpointed id returns ZMC_ECLOSED or ZMC_ENOTFOUND. */
zmc_status zmc_checkpoint(zmc_ctx *ctx, uint64_t job_id, zmc_moments *out, int32_t wait_ms);

/* Submit a job that continues from moments taken earlier (a zmc_checkpoint, or
 * zmc_integrate_moments over samples [0, from[i].n) of the same stream):
 * integrand i samples [from[i].n, desc[i].n_samples) of its stream and its
 * result combines from[i] with them (Chan's pairwise update on the device), so
 * that it equals an uninterrupted run of desc[i] up to FP64 rounding of the
 * merge.  Needs from[i].n <= desc[i].n_samples and from[i].n a multiple of 5 or
 * equal to n_samples (ZMC_EINVAL otherwise); from[i].n = 0 starts afresh.
 * Otherwise as zmc_submit. */
zmc_status zmc_submit_resume(zmc_ctx *ctx, const zmc_desc *desc, const zmc_moments *from,
                             size_t n, uint64_t *job_id);

/* Ids of jobs that finished (done, failed or cancelled) since the last call, up
 * to cap of them, into job_ids (host array); *n_out is the count.  Each finished
 * job is reported once; collect its results with zmc_poll.  wait_ms as in
 * zmc_poll (ZMC_EAGAIN / ZMC_ETIMEOUT when none finished). */
zmc_status zmc_poll_any(zmc_ctx *ctx, uint64_t *job_ids, size_t cap, int32_t wait_ms,
                        size_t *n_out);

zmc_status zmc_serving_stats_get(zmc_ctx *ctx, zmc_serving_stats *out);

/* Device-resident plan: the descriptor table precomputed and uploaded once,
 * its partial-sum records and results kept in the arena, so the sampling and
 * merge launches can be replayed (as a CUDA graph) without host traffic. */
zmc_status zmc_plan_create(zmc_ctx *ctx, const zmc_desc *desc, size_t n, zmc_plan **out);

#define ZMC_STAGE_SAMPLE 1u /* reset the work counter + persistent sampling launch */
#define ZMC_STAGE_MERGE 2u  /* FP64 merge of every integrand's chunk records       */
#define ZMC_STAGE_ALL 3u    /* both, replayed as one captured CUDA graph           */

/* Enqueue the chosen stages on the context stream; returns without waiting. */
zmc_status zmc_plan_run(zmc_plan *plan, uint32_t stages);

/* Enqueue the plain FP64 form (one launch per integrand + merge). */
zmc_status zmc_plan_run_plain(zmc_plan *plan);

/* Wait for the stream and copy the plan's n results to the host. */
zmc_status zmc_plan_results(zmc_plan *plan, zmc_result *out);

/* Device pointer to the plan's results (n zmc_result rows). */
zmc_status zmc_plan_device_results(zmc_plan *plan, void **device_ptr);

zmc_status zmc_plan_info_get(const zmc_plan *plan, zmc_plan_info *out);
zmc_status zmc_plan_destroy(zmc_plan *plan);

/* Philox4x32-10 of n counters (host array, n x 4 words) under n keys (n x 2),
 * computed by the same device routine the sampling kernel uses; out is n x 4. */
zmc_status zmc_philox4x32_10(zmc_ctx *ctx, const uint32_t *ctr, const uint32_t *key,
                             uint32_t *out, size_t n);

/* Throughput of the generator alone on the context's device: Philox4x32-10
 * blocks per second (into *blocks_per_second) of a kernel that only draws
 * blocks, with the sampling kernels' counter layout and launch bound (one wave
 * of 2 x 256-thread blocks per SM, four independent calls at a time per
 * thread), timed with CUDA events on the context's stream after one untimed
 * launch.  n_blocks (1..2^40) is rounded up to a whole number of groups of 4
 * per thread.  The paper has no counterpart; it measures the ceiling of every
 * sampling kernel, which draws d / 5 blocks per d-dimensional sample.
 * ZMC_EINVAL for n_blocks out of range, ZMC_ENOMEM if the arena cannot hold
 * one word per thread, ZMC_ECUDA on a CUDA error. */
zmc_status zmc_philox_rate(zmc_ctx *ctx, uint64_t n_blocks, double *blocks_per_second);

/* FP32 values f(x_s) of samples s in [s_begin, s_begin + count) of one
 * integrand, computed by the sampling kernel's own generation, map and
 * evaluation code; out has count floats (host). */
zmc_status zmc_eval_samples(zmc_ctx *ctx, const zmc_desc *desc, uint64_t s_begin,
                            uint32_t count, float *out);

/* ---- User-defined integrands, compiled at run time ----------------------------
 * The paper's integrators take the integrand as a user-written function that
 * is compiled for the GPU (Sec. "Summary of revisions" and "Solution method":
 * the multi-function mode integrates functions of different forms, dimensions
 * and domains).  zmc_udf_create compiles `source` (CUDA C++, NUL-terminated) with
 * NVRTC for this GPU; the source must define, for precision ZMC_UDF_F32:
 *     __device__ float  zmc_user_f(const float *x, const float *p)
 * or, for ZMC_UDF_F64:
 *     __device__ double zmc_user_f(const double *x, const double *p)
 * x is the sample point (dim coordinates, dim 1..12), p the descriptor's ZMC_NPARAM
 * parameters (zmc_desc.p, rounded to float for ZMC_UDF_F32).  The macros
 * ZMC_UDF_DIM and ZMC_UDF_PRECISION are defined for the source.  The library
 * supplies the rest of the path -- the same Philox4x32-10 words and box map as
 * the built-in families (so a user form of a built-in integrand sees exactly
 * the same samples), FP32 per-chunk sums of S f and the FP64 merge.
 *   ZMC_UDF_F32: map x_i = lo_i + w_i u_i and f in FP32 (fastest; the user's
 *                FP32 arithmetic decides the accuracy of f).
 *   ZMC_UDF_F64: map and f in FP64, each value rounded to FP32 before the sums
 *                (relative error 2^-24 per sample; slower on GB300's FP64 rate).
 * `amplitude` > 0 is an upper bound of |f| over every box the udf integrates;
 * the library then sums S f with S = 2^(48 - ceil(log2 amplitude)) so that
 * values down to ~2^-111 amplitude keep their squares in FP32 range (0: S = 1,
 * fine for |f| within about [1e-18, 1e18]).
 * Returns ZMC_EINVAL with the start of the compiler log in zmc_last_error() if
 * the source does not compile, ZMC_ENOSYS if NVRTC cannot be loaded.  Needs no
 * GPU and no context; the compiled image is loaded on a device at first use.  */
#define ZMC_UDF_F32 0u
#define ZMC_UDF_F64 1u
typedef struct zmc_udf zmc_udf;
zmc_status zmc_udf_create(const char *source, uint32_t dim, uint32_t precision,
                          double amplitude, zmc_udf **out);

/* Several user integrands, each of its own form and dimension, in one module
 * (the multi-function mode with user code: one launch integrates rows of all of
 * them).  Function k is sources[k] (each defines its own zmc_user_f; the sources
 * are compiled in separate namespaces, so helper names may repeat), of dimension
 * dims[k] and bound amplitudes[k] (amplitudes may be NULL: all 0).  1 <= n_funcs
 * <= 64; one precision for all.  A row selects function k with desc.deg = k.
 * Errors name the failing source as zmc_user_source_<k>. */
zmc_status zmc_udf_create_multi(const char *const *sources, const uint32_t *dims,
                                uint32_t n_funcs, uint32_t precision, const double *amplitudes,
                                zmc_udf **out);

/* Integrate n descriptors (host array) with compiled user integrands: every
 * desc[i].family must be ZMC_USER, desc[i].deg selects the function (0 for a
 * udf of one function) and desc[i].dim must be that function's dimension, at
 * most 7 here (box, samples, seed, stream and p as for the built-in families;
 * functions of 8 to 12 dimensions integrate through zmc_normal_integrate_udf).
 * Results (host array) as zmc_integrate's.  Blocking, on the context's stream. */
zmc_status zmc_udf_integrate(zmc_ctx *ctx, const zmc_udf *udf, const zmc_desc *desc,
                             size_t n, zmc_result *out);

/* FP32 values f(x_s), s in [s_begin, s_begin + count), of one descriptor, from
 * the same generation, map and evaluation as zmc_udf_integrate (for tests). */
zmc_status zmc_udf_eval_samples(zmc_ctx *ctx, const zmc_udf *udf, const zmc_desc *desc,
                                uint64_t s_begin, uint32_t count, float *out);

/* The NVRTC log of the udf's compilation (warnings; "" if none). */
const char *zmc_udf_log(const zmc_udf *udf);

/* Release a udf (NULL accepted).  Not while a call using it is running. */
zmc_status zmc_udf_destroy(zmc_udf *udf);

/* ---- Stratified sampling with a heuristic tree search (ZMCintegral_normal) -----
 * The paper's normal mode (Sec. "Solution method", "Additional comments": for
 * integrands of higher dimension, 8 to 12) stratifies the domain and refines
 * the strata by a heuristic tree search; it gives no steps, and these calls
 * implement this reading of it:
 *   1. the box is cut into divisions^dim equal cells (cell j has grid index
 *      (j / divisions^i) mod divisions in dimension i);
 *   2. every cell is integrated by direct Monte Carlo with samples_per_cell
 *      samples; the j-th cell created uses Philox stream stream_base + j and key
 *      seed; e_c = V_c mean_c, s_c = V_c sqrt(M2_c / (N_c (N_c - 1)));
 *   3. up to `depth` times: with tau = sigma_mult * (mean of s_c over the leaves),
 *      every leaf with s_c > tau is split into its 2^dim halves (child b takes
 *      the upper half of dimension i when bit i of b is set; mid = lo + (hi - lo)/2),
 *      in leaf order while the leaf count stays <= max_leaves; the children take
 *      their parent's place in the leaf order and are integrated as in step 2;
 *      a round that splits nothing ends the search;
 *   4. estimate = sum of e_c over the leaves, stderr = sqrt(sum of s_c^2).
 * Cell boundaries: lo_i + ((hi_i - lo_i) * idx) / divisions, the last one hi_i. */
typedef struct zmc_normal_opts {
    uint32_t divisions;        /* cells per dimension at level 0 (>= 1; divisions^dim <= 2^20) */
    uint32_t depth;            /* refinement rounds at most (0: plain stratified sampling)    */
    uint64_t samples_per_cell; /* samples of every cell (2 .. 2^40)                           */
    double sigma_mult;         /* split threshold factor (> 0)                                */
    uint64_t seed;             /* Philox key of every cell                                    */
    uint32_t stream_base;      /* stream of the first cell                                    */
    uint32_t max_leaves;       /* cap on the leaf count (0: 2^20; at most 2^22)               */
} zmc_normal_opts;

typedef struct zmc_normal_result {
    double estimate;
    double stderr_;
    uint64_t n_samples;        /* samples taken over every cell evaluated                     */
    uint64_t n_cells;          /* cells evaluated (split ones included)                       */
    uint64_t n_leaves;         /* cells of the final partition                                */
    uint32_t rounds;           /* refinement rounds that split at least one leaf              */
    int32_t status;
} zmc_normal_result;

/* divisions 2, depth 2, 2^14 samples per cell, sigma_mult 2, seed 0, stream 0,
 * max_leaves 2^20. */
zmc_status zmc_normal_default_options(zmc_normal_opts *opt);

/* A built-in family integrand: base gives family, dim (<= 7), box and p; its
 * n_samples, seed and stream_id are replaced by the options.  Blocking. */
zmc_status zmc_normal_integrate(zmc_ctx *ctx, const zmc_desc *base, const zmc_normal_opts *opt,
                                zmc_normal_result *out);

/* A user-defined integrand of any dimension the udf was compiled for (1..12;
 * function 0 of a multi-function udf): lo, hi (its dim values each) give the
 * box, p the ZMC_NPARAM parameters. */
zmc_status zmc_normal_integrate_udf(zmc_ctx *ctx, const zmc_udf *udf, const double *lo,
                                    const double *hi, const double *p,
                                    const zmc_normal_opts *opt, zmc_normal_result *out);

/* ---- Integration without allocation (the paper has no counterpart) -------------
 * For callers that must not allocate device memory when they need a result: a
 * framework whose pool owns all device memory and forbids side allocations, a
 * latency-bound loop that cannot take an allocation's implicit synchronisation
 * or its failure on a nearly full device, or code that cannot create a context
 * (zmc_create allocates an arena).
 *
 * zmc_integrate_noalloc computes what zmc_integrate computes for desc[0..n) (host
 * array) and writes the n results to `out`, a DEVICE array the caller owns.  It
 * is asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream) on
 * the current device: read `out` after synchronising the stream.  It needs no
 * context and allocates nothing: its launch header, work list, device
 * descriptors and partial sums live in one fixed array of
 * ZMC_NOALLOC_SCRATCH_BYTES compiled into the library.  A device reserves the
 * array once the library's device code is loaded there (with CUDA's lazy module
 * loading, at the latest on the first call on that device) and holds it until
 * the process exits.
 *   - At most ZMC_NOALLOC_MAX_FNS integrands (ZMC_EINVAL beyond) and at most
 *     ~3.4e10 samples in total at 16640 samples per chunk (ZMC_ENOMEM beyond, with
 *     the needed size in zmc_last_error()).
 *   - All calls share the array and it keeps the previous call's contents; each
 *     call re-uploads its tables and zeroes its work counters.  Calls whose GPU
 *     work overlaps (other streams, or unordered host threads) race: order them.
 *   - The tables are uploaded from a static host buffer.  Before a call
 *     rewrites it, the call waits until the previous call's upload has run on
 *     the GPU, so a call may block until the previous call's stream reaches
 *     that upload.
 *   - The first call on a device looks up the array's device address and
 *     creates one event (no memory allocation) with that device current; make
 *     it before any stream capture.
 *   - Results equal zmc_integrate's with the default quints_per_lane (104).     */
#define ZMC_NOALLOC_SCRATCH_BYTES (16u << 20)
#define ZMC_NOALLOC_MAX_FNS 4096u
zmc_status zmc_integrate_noalloc(const zmc_desc *desc, size_t n, zmc_result *out,
                                 void *stream);

/* Host-only check of n descriptors with the rules listed at zmc_desc (no GPU
 * needed).  Returns ZMC_OK, or ZMC_EINVAL with *bad_index (if non-NULL) set to
 * the first rejected row. */
zmc_status zmc_validate(const zmc_desc *desc, size_t n, size_t *bad_index);

/* Host-only inspection (no GPU needed): the evaluation form the library picks
 * for each of n descriptors, written to forms[i] as
 *     (form << 8) | (family << 4) | dim,
 * with form, by family:
 *   ZMC_HARMONIC  0 general phase; 1 equal phase rates in every dimension
 *                 (dim >= 2 and every k_i (hi_i - lo_i) the same after rounding
 *                 to 2^-41 turn): the phase through the sum of the coordinates
 *   ZMC_ABSLIN    0 c.x summed in 64-bit integers; 1 in 32-bit integers (rows of
 *                 >= 256 samples)
 *   ZMC_GAUSS     0 mu within [-1, 2] box widths of lo in every dimension; 1 not
 *   ZMC_POLY      deg (0..4): coefficient form; deg + 3 (5..7): factors in
 *                 root form (degrees 2..4)
 * Rows the rules of zmc_desc reject give ZMC_EINVAL and *bad_index (if not
 * NULL), as zmc_validate.  Forms never change what is integrated, only how
 * (tests use this to check that their tables reach every form). */
zmc_status zmc_variant_of(const zmc_desc *desc, size_t n, uint32_t *forms, size_t *bad_index);

/* The serving scheduler's rule for filling one persistent launch (host only; no
 * GPU or context needed, so the rule can be checked anywhere).  Job i is the
 * i-th oldest live job and has chunks_left[i] chunks of chunk_samples samples
 * left to issue; on return take[i] holds the chunks it contributes to a launch
 * of at most budget chunks (sum take <= budget, take[i] <= chunks_left[i]).
 *   share == 0 (oldest first): each job in turn takes its remaining chunks up
 *     to what is left of the budget; if the backlog, sum chunks_left[i] *
 *     chunk_samples, is below cut_backlog, the launch ends with the first job
 *     it completes (cut_backlog 0: never);
 *   share > 0 (equal shares): passes over the jobs with work left, each taking
 *     up to max(share, budget left / jobs with work left) per pass, until the
 *     budget or the work runs out.
 * Layouts: chunks_left and take hold n_jobs values (caller-owned).  Errors:
 * ZMC_EINVAL for a NULL array with n_jobs > 0 or chunk_samples == 0. */
zmc_status zmc_serving_fill(const uint64_t *chunks_left, size_t n_jobs, uint64_t budget,
                            uint32_t share, uint64_t cut_backlog, uint64_t chunk_samples,
                            uint64_t *take);

/* sizeof checks for foreign-language bindings. */
size_t zmc_desc_size(void);
size_t zmc_result_size(void);

#ifdef __cplusplus
}
#endif
#endif /* ZMC_H */
