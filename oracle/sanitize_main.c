/*
 * TEST INFRASTRUCTURE ONLY: a standalone driver that runs the oracle's
 * routines on small synthetic inputs, for building with the address and
 * undefined-behaviour sanitizers (tests/test_oracle_sanitizers.py).  It
 * includes the oracle's source, so that one compilation unit is checked,
 * and prints one line per case; any sanitizer report fails the test.
 */
#include <stdio.h>
#include <stdlib.h>

#include "gmmsp_oracle.c"

static unsigned long long rng_state = 88172645463325252ull;

static double uniform(double lo, double hi)
{
    /* xorshift64 (Marsaglia 2003) */
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return lo + (hi - lo) * (double)(rng_state >> 11) / 9007199254740992.0;
}

static int run_case(int W, int H, int K_req, int spacing, int T, int cmodel)
{
    int g[4], rc;
    long N = (long)W * H, i;
    double *lab, *mu, *cs, *cc, *margin, *loglik;
    int32_t *labels;
    int raised[64];
    if (orc_grid(W, H, K_req, spacing, g)) return -1;
    lab = malloc(sizeof(double) * 3 * N);
    mu = malloc(sizeof(double) * 5 * g[3]);
    cs = malloc(sizeof(double) * 3 * g[3]);
    cc = malloc(sizeof(double) * 6 * g[3]);
    margin = malloc(sizeof(double) * N);
    loglik = malloc(sizeof(double) * (T + 1));
    labels = malloc(sizeof(int32_t) * N);
    for (i = 0; i < N; ++i) {
        lab[3 * i + 0] = uniform(0.0, 100.0);
        lab[3 * i + 1] = uniform(-60.0, 60.0);
        lab[3 * i + 2] = uniform(-60.0, 60.0);
    }
    rc = orc_em(lab, W, H, K_req, spacing, T, 8.0, 2.0, 8.0, NULL, NULL, NULL, mu, cs, cc, labels, margin,
                loglik, NULL, NULL, NULL, raised, cmodel);
    printf("W=%d H=%d v=%d K=%d T=%d model=%d rc=%d L=%.6f\n", W, H, g[0], g[3], T, cmodel, rc, loglik[T]);
    free(lab); free(mu); free(cs); free(cc); free(margin); free(loglik); free(labels);
    return rc < 0 ? rc : 0;
}

int main(void)
{
    const int cases[][5] = {{16, 16, 0, 4, 3}, {37, 23, 0, 6, 5}, {19, 17, 0, 5, 4}, {40, 30, 12, 0, 3}};
    int c, m;
    uint8_t rgb[3 * 64], gray[64];
    double out[3 * 64];
    orc_set_threads(1);
    for (c = 0; c < 4; ++c)
        for (m = 0; m < 3; ++m)
            if (run_case(cases[c][0], cases[c][1], cases[c][2], cases[c][3], cases[c][4], m)) return 1;
    for (c = 0; c < 3 * 64; ++c) rgb[c] = (uint8_t)(c * 37);
    for (c = 0; c < 64; ++c) gray[c] = (uint8_t)(c * 4);
    orc_rgb2lab(rgb, 64, out);
    orc_gray2l(gray, 64, out);
    printf("ok\n");
    return 0;
}
