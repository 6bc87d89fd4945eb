/*
 * zmc_oracle.c -- plain, slow, FP64 CPU oracle for multi-function direct Monte
 * Carlo integration (ZMCintegral-v5.1, arXiv 2104.10073).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * constant table or helper with the CUDA implementation, and the product path
 * never calls it.
 *
 * What it computes, step by step in the order the method states them:
 *
 *   Sec. "Solution method": each integrand gets its own direct Monte Carlo
 *   estimate.  For integrand f over the box B = prod_i [lo_i, hi_i] with
 *   N samples x_s drawn uniformly on B,
 *
 *       mean     = (1/N) sum_s f(x_s)
 *       estimate = V * mean,                  V = prod_i (hi_i - lo_i)
 *       stderr   = V * sqrt(M2 / (N (N-1))),  M2 = sum_s (f(x_s) - mean)^2
 *
 *   (the paper shows mean and spread of repeated estimates, Fig. 1 caption;
 *   the per-run standard error with the N-1 denominator is the reading taken
 *   for the spread of one run).  mean and M2 are accumulated with Welford's
 *   one-sample update in FP64, in sample order.
 *
 *   Sampling: integrand f (key = seed, stream = stream_id) consumes the field
 *   stream c = s*d + i (sample s, coordinate i).  Field c is the 23-bit field
 *   k = c mod 5, bits 23k .. 23k+22, of block b = c div 5, where a block is the
 *   128-bit output of Philox4x32-10 applied to counter (stream_id, b mod 2^32,
 *   b div 2^32, 0) with key (seed mod 2^32, seed div 2^32), read as one number
 *   with its word 0 least significant (five fields per block; its top 13 bits
 *   are not used).  Philox4x32-10 is the generator of Salmon, Moraes, Dror and
 *   Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
 *   the 4x32 S-box with the two published multipliers, the key bumped by the
 *   two published Weyl constants between rounds.  A field r gives
 *   u = r * 2^-23 in [0, 1), exact in binary64, and x_i = lo_i + (hi_i - lo_i) u_i.
 *
 *   Integrand families, evaluated directly in FP64 with libm:
 *     HARMONIC  a cos(k.x) + b sin(k.x)                      (Eq. 1)
 *     ABSLIN    a |c.x|                                      (Eq. 2)
 *     GAUSS     A exp(-|x - mu|^2 / (2 sigma^2))
 *     POLY      prod_i sum_{j<=deg} c_ij x_i^j
 *
 * Descriptor columns (one entry per integrand; lo, hi hold 7 doubles per row,
 * p holds 40):
 *   HARMONIC p[0]=a p[1]=b p[2+i]=k_i;  ABSLIN p[0]=a p[1+i]=c_i;
 *   GAUSS p[0]=A p[1]=sigma p[2+i]=mu_i;  POLY p[5i+j]=c_ij, j <= deg.
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused multiply-add contraction,
 * so the oracle gives the same bits on every host), optional OpenMP over
 * integrands.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ZO_MAX_DIM 7
#define ZO_NPARAM 40

/* ---------------------------------------------------------------- Philox4x32-10
 * Round function and key schedule as published by Salmon et al. (SC'11). */
#define ZO_PHILOX_M0 0xD2511F53u
#define ZO_PHILOX_M1 0xCD9E8D57u
#define ZO_PHILOX_W0 0x9E3779B9u
#define ZO_PHILOX_W1 0xBB67AE85u

static void zo_philox_round(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    uint64_t prod0 = (uint64_t)ZO_PHILOX_M0 * (uint64_t)c[0];
    uint64_t prod1 = (uint64_t)ZO_PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
}

void zo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        zo_philox_round(c, k0, k1);
        k0 += ZO_PHILOX_W0;
        k1 += ZO_PHILOX_W1;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* n independent calls: ctr is n x 4, key is n x 2, out is n x 4 (row major). */
void zo_philox_many(size_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    for (size_t j = 0; j < n; ++j)
        zo_philox4x32_10(ctr + 4 * j, key + 2 * j, out + 4 * j);
}

/* ---------------------------------------------------------------- one integrand */
typedef struct {
    uint32_t family, dim, stream_id, deg;
    uint64_t n_samples, seed;
    const double *lo, *hi, *p;
} zo_fn;

/* Field c of an integrand's stream, with a one-block cache (c increases). */
typedef struct {
    uint64_t block;
    int valid;
    uint32_t words[4];
} zo_cache;

static uint32_t zo_field(const zo_fn *f, uint64_t c, zo_cache *cache)
{
    uint64_t b = c / 5;
    if (!cache->valid || cache->block != b) {
        uint32_t ctr[4] = {f->stream_id, (uint32_t)b, (uint32_t)(b >> 32), 0u};
        uint32_t key[2] = {(uint32_t)f->seed, (uint32_t)(f->seed >> 32)};
        zo_philox4x32_10(ctr, key, cache->words);
        cache->block = b;
        cache->valid = 1;
    }
    /* bits 23k .. 23k+22 of the block, one bit at a time: block bit q is bit
       q mod 32 of word q div 32 */
    uint32_t first = 23u * (uint32_t)(c % 5);
    uint32_t r = 0;
    for (uint32_t j = 0; j < 23; ++j) {
        uint32_t q = first + j;
        r |= ((cache->words[q / 32] >> (q % 32)) & 1u) << j;
    }
    return r;
}

static double zo_uniform(uint32_t r)
{
    return (double)(r & 0x7FFFFFu) * (1.0 / 8388608.0); /* 2^-23 */
}

static double zo_eval(const zo_fn *f, const double *x)
{
    const double *p = f->p;
    int d = (int)f->dim;
    switch (f->family) {
    case 0: { /* HARMONIC, Eq. 1 */
        double phase = 0.0;
        for (int i = 0; i < d; ++i)
            phase += p[2 + i] * x[i];
        return p[0] * cos(phase) + p[1] * sin(phase);
    }
    case 1: { /* ABSLIN, Eq. 2 */
        double s = 0.0;
        for (int i = 0; i < d; ++i)
            s += p[1 + i] * x[i];
        return p[0] * fabs(s);
    }
    case 2: { /* GAUSS */
        double r2 = 0.0;
        for (int i = 0; i < d; ++i) {
            double t = x[i] - p[2 + i];
            r2 += t * t;
        }
        return p[0] * exp(-r2 / (2.0 * p[1] * p[1]));
    }
    case 3: { /* POLY */
        double prod = 1.0;
        for (int i = 0; i < d; ++i) {
            double acc = 0.0, xp = 1.0;
            for (int j = 0; j <= (int)f->deg; ++j) {
                acc += p[5 * i + j] * xp;
                xp *= x[i];
            }
            prod *= acc;
        }
        return prod;
    }
    default:
        return NAN;
    }
}

/* Point x of sample s (and its d raw 23-bit fields). */
static void zo_point(const zo_fn *f, uint64_t s, zo_cache *cache, uint32_t *words, double *x)
{
    for (uint32_t i = 0; i < f->dim; ++i) {
        uint32_t r = zo_field(f, s * (uint64_t)f->dim + i, cache);
        if (words)
            words[i] = r;
        x[i] = f->lo[i] + (f->hi[i] - f->lo[i]) * zo_uniform(r);
    }
}

static double zo_volume(const zo_fn *f)
{
    double v = 1.0;
    for (uint32_t i = 0; i < f->dim; ++i)
        v *= f->hi[i] - f->lo[i];
    return v;
}

/* Welford moments of f over samples [s_begin, s_end). */
static void zo_moments_fn(const zo_fn *f, uint64_t s_begin, uint64_t s_end, double *n_out,
                          double *mean_out, double *m2_out, double *sum_abs_out)
{
    zo_cache cache = {0, 0, {0, 0, 0, 0}};
    double x[ZO_MAX_DIM];
    double n = 0.0, mean = 0.0, m2 = 0.0, sum_abs = 0.0;
    for (uint64_t s = s_begin; s < s_end; ++s) {
        zo_point(f, s, &cache, NULL, x);
        double v = zo_eval(f, x);
        n += 1.0;
        double delta = v - mean;
        mean += delta / n;
        m2 += delta * (v - mean);
        sum_abs += fabs(v);
    }
    *n_out = n;
    *mean_out = mean;
    *m2_out = m2;
    *sum_abs_out = sum_abs;
}

static zo_fn zo_row(size_t j, const uint32_t *family, const uint32_t *dim,
                    const uint32_t *stream_id, const uint32_t *deg, const uint64_t *n_samples,
                    const uint64_t *seed, const double *lo, const double *hi, const double *p)
{
    zo_fn f;
    f.family = family[j];
    f.dim = dim[j];
    f.stream_id = stream_id[j];
    f.deg = deg[j];
    f.n_samples = n_samples[j];
    f.seed = seed[j];
    f.lo = lo + ZO_MAX_DIM * j;
    f.hi = hi + ZO_MAX_DIM * j;
    f.p = p + ZO_NPARAM * j;
    return f;
}

/*
 * Integrate n_fn integrands.  Outputs per row: estimate, stderr (NaN for N = 1),
 * mean |f| (the scale the parity tolerance is stated against) and N.
 * threads <= 0 uses the OpenMP default.  Returns the number of threads used.
 */
int zo_integrate(size_t n_fn, const uint32_t *family, const uint32_t *dim,
                 const uint32_t *stream_id, const uint32_t *deg, const uint64_t *n_samples,
                 const uint64_t *seed, const double *lo, const double *hi, const double *p,
                 double *estimate, double *stderr_out, double *mean_abs, int threads)
{
    int used = 1;
#ifdef _OPENMP
    if (threads > 0)
        omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long long jj = 0; jj < (long long)n_fn; ++jj) {
        size_t j = (size_t)jj;
        zo_fn f = zo_row(j, family, dim, stream_id, deg, n_samples, seed, lo, hi, p);
        double n, mean, m2, sum_abs;
        zo_moments_fn(&f, 0, f.n_samples, &n, &mean, &m2, &sum_abs);
        double v = zo_volume(&f);
        estimate[j] = v * mean;
        stderr_out[j] = v * sqrt(m2 / (n * (n - 1.0)));
        mean_abs[j] = sum_abs / n;
    }
    return used;
}

/* Welford moments (n, mean, M2, sum |f|) of one integrand over [s_begin, s_end). */
void zo_moments(uint32_t family, uint32_t dim, uint32_t stream_id, uint32_t deg,
                uint64_t seed, const double *lo, const double *hi, const double *p,
                uint64_t s_begin, uint64_t s_end, double *out4)
{
    zo_fn f = {family, dim, stream_id, deg, s_end, seed, lo, hi, p};
    zo_moments_fn(&f, s_begin, s_end, &out4[0], &out4[1], &out4[2], &out4[3]);
}

/* Raw 23-bit fields (count x dim), points (count x dim) and values (count) of samples
 * [s_begin, s_begin + count) of one integrand. */
void zo_samples(uint32_t family, uint32_t dim, uint32_t stream_id, uint32_t deg,
                uint64_t seed, const double *lo, const double *hi, const double *p,
                uint64_t s_begin, uint64_t count, uint32_t *words, double *x, double *fx)
{
    zo_fn f = {family, dim, stream_id, deg, s_begin + count, seed, lo, hi, p};
    zo_cache cache = {0, 0, {0, 0, 0, 0}};
    for (uint64_t t = 0; t < count; ++t) {
        zo_point(&f, s_begin + t, &cache, words + t * dim, x + t * dim);
        fx[t] = zo_eval(&f, x + t * dim);
    }
}
