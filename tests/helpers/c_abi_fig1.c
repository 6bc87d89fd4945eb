/* Plain C user of the library's C ABI (no Python, no C++): integrates the Fig. 1
 * harmonics (Eq. 1, n = 1..100, k_n = (n+50)/(2 pi) in all four dimensions,
 * [0,1]^4) with zmc_integrate and through the serving calls, and prints one
 * line per integrand: n, estimate, stderr (blocking call) and estimate (served).
 * Exit status: 0 on success, 1 on any library error (message on stderr). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "zmc.h"

static int fail(const char *what, zmc_status st) {
    fprintf(stderr, "%s: status %d: %s\n", what, (int)st, zmc_last_error(NULL));
    return 1;
}

int main(int argc, char **argv) {
    const uint64_t n_samples = argc > 1 ? strtoull(argv[1], NULL, 10) : 100000u;
    const double two_pi = 6.283185307179586476925286766559;
    zmc_desc desc[100];
    memset(desc, 0, sizeof desc);
    for (int n = 1; n <= 100; ++n) {
        zmc_desc *d = &desc[n - 1];
        d->family = ZMC_HARMONIC;
        d->dim = 4;
        d->stream_id = (uint32_t)(n - 1);
        d->n_samples = n_samples;
        d->seed = 0;
        d->p[0] = 1.0;
        d->p[1] = 1.0;
        for (int i = 0; i < 4; ++i) {
            d->lo[i] = 0.0;
            d->hi[i] = 1.0;
            d->p[2 + i] = (n + 50) / two_pi;
        }
    }
    zmc_options opt;
    zmc_status st = zmc_default_options(&opt);
    if (st != ZMC_OK) return fail("zmc_default_options", st);
    opt.mem_budget_bytes = 256u << 20;
    opt.serving = 1;
    zmc_ctx *ctx = NULL;
    st = zmc_create(&opt, &ctx);
    if (st != ZMC_OK) return fail("zmc_create", st);
    zmc_result res[100], served[100];
    st = zmc_integrate(ctx, desc, 100, res);
    if (st != ZMC_OK) return fail("zmc_integrate", st);
    uint64_t job = 0;
    st = zmc_submit(ctx, desc, 100, &job);
    if (st != ZMC_OK) return fail("zmc_submit", st);
    st = zmc_poll(ctx, job, served, 60000);
    if (st != ZMC_OK) return fail("zmc_poll", st);
    for (int n = 1; n <= 100; ++n)
        printf("%d %.17g %.17g %.17g\n", n, res[n - 1].estimate, res[n - 1].stderr_,
               served[n - 1].estimate);
    st = zmc_destroy(ctx);
    if (st != ZMC_OK) return fail("zmc_destroy", st);
    return 0;
}
