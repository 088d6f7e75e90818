/*
 * sanitize_oracle.c -- drives every entry point of the CPU oracle on small inputs, for a build
 * with AddressSanitizer and UndefinedBehaviorSanitizer (tests/test_oracle_sanitize.py compiles
 * and runs it).  Every buffer is allocated at exactly the size the oracle's header states, so an
 * out-of-bounds access, a use of freed memory or undefined arithmetic aborts the run.  The
 * inputs cover the degenerate orders (0, 1, 2), exact zeros in e (splits), coincident
 * eigenvalues (glued W21+ blocks) and a cluster large enough to exercise every orthogonalizer.
 * Prints "ok" and exits 0 when nothing was reported.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "../oracle/tinv_oracle.h"

static double* dalloc(int64_t k)
{
    return (double*)malloc((size_t)(k > 0 ? k : 1) * sizeof(double));
}

/* glued Wilkinson: g blocks of W21+ (d_i = |10 - i|, e = 1 inside a block), glue e = glue */
static int64_t glued(int g, double glue, double** d, double** e)
{
    const int64_t n = 21 * (int64_t)g;
    *d = dalloc(n);
    *e = dalloc(n - 1);
    for (int64_t i = 0; i < n; ++i) (*d)[i] = fabs(10.0 - (double)(i % 21));
    for (int64_t i = 0; i + 1 < n; ++i) (*e)[i] = ((i + 1) % 21 == 0) ? glue : 1.0;
    return n;
}

static void uniform(int64_t n, uint64_t seed, double* d, double* e)
{
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) d[i] = 2.0 * ((double)(orc_sm64_next(&s) >> 11) * 0x1p-53) - 1.0;
    for (int64_t i = 0; i + 1 < n; ++i) e[i] = 2.0 * ((double)(orc_sm64_next(&s) >> 11) * 0x1p-53) - 1.0;
}

/* the whole path on one matrix: split, bisection, plan, LU and solve of one shift, inverse
 * iteration with each method, and the dense Jacobi check for small n */
static void run_path(int64_t n, const double* d, const double* e)
{
    int64_t* isplit = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    (void)orc_split(n, d, e, isplit);
    (void)orc_onenorm(n, d, e);
    double* w = dalloc(n);
    orc_bisect(n, d, e, w);
    (void)orc_sturm_count(n, d, e, n > 0 ? w[n / 2] : 0.0, 1e-300);
    double* wp = dalloc(n);
    int64_t* head = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    double onenrm, ortol, dtpcrt;
    orc_plan(n, d, e, n, w, wp, head, &onenrm, &ortol, &dtpcrt);
    if (n > 0) {
        double *u0 = dalloc(n), *u1 = dalloc(n), *u2 = dalloc(n), *l = dalloc(n), *y = dalloc(n);
        unsigned char* piv = (unsigned char*)malloc((size_t)n);
        orc_lagtf(n, d, e, wp[0], u0, u1, u2, l, piv);
        for (int64_t i = 0; i < n; ++i) y[i] = orc_start_value(7, 0, 0, i);
        (void)orc_lagts(n, u0, u1, u2, l, piv, y);
        free(u0), free(u1), free(u2), free(l), free(y), free(piv);
    }
    for (int method = ORC_MGS; method <= ORC_HOUSE; ++method) {
        double* Z = dalloc(n * n);
        int64_t* ifail = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        int32_t* iters = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        orc_stats st;
        (void)orc_tinv(n, d, e, n, w, 0, Z, n > 0 ? n : 1, method, 3, ifail, iters, &st);
        /* a sub-range with its offset, as the tests use it */
        if (n >= 4) (void)orc_tinv(n, d, e, 2, w + n / 2, n / 2, Z, n, method, 3, ifail, iters, NULL);
        if (method == ORC_CWY) {
            (void)orc_tinv_blocked(n, d, e, n, w, 0, Z, n > 0 ? n : 1, 4, 3, ifail, iters, &st);
            if (n >= 4) (void)orc_tinv_blocked(n, d, e, 2, w + n / 2, n / 2, Z, n, 3, 3, ifail, iters, NULL);
        }
        free(Z), free(ifail), free(iters);
    }
    if (n > 0 && n <= 64) {
        double *A = dalloc(n * n), *lam = dalloc(n), *V = dalloc(n * n);
        for (int64_t i = 0; i < n * n; ++i) A[i] = 0.0;
        for (int64_t i = 0; i < n; ++i) A[i + i * n] = d[i];
        for (int64_t i = 0; i + 1 < n; ++i) A[i + 1 + i * n] = A[i + (i + 1) * n] = e[i];
        orc_jacobi(n, A, lam, V);
        free(A), free(lam), free(V);
    }
    free(isplit), free(w), free(wp), free(head);
}

/* the stand-alone orthogonalizers on an n x m block with a leading dimension larger than n */
static void run_orth(int64_t n, int64_t m)
{
    const int64_t ld = n + 3;
    double *V = dalloc(ld * m), *Q = dalloc(ld * m), *Y = dalloc(n * m), *T = dalloc(m * m),
           *tv = dalloc(m);
    for (int64_t j = 0; j < m; ++j)
        for (int64_t i = 0; i < ld; ++i) V[i + j * ld] = orc_start_value(11, j, 0, i);
    (void)orc_orth_mgs(n, m, V, ld, Q, ld);
    (void)orc_orth_house(n, m, V, ld, Q, ld, Y, tv);
    (void)orc_orth_cwy_ordinary(n, m, V, ld, Q, ld, Y, T);
    (void)orc_orth_cwy_new(n, m, V, ld, Q, ld, Y, T);
    (void)orc_orth_house(n, m, V, ld, Q, ld, NULL, NULL);
    (void)orc_orth_cwy_new(n, m, V, ld, Q, ld, NULL, NULL);
    (void)orc_orth_cwy_block(n, m, V, ld, 3, Q, ld, Y, T);
    (void)orc_orth_cwy_block(n, m, V, ld, m + 2, Q, ld, NULL, NULL);
    free(V), free(Q), free(Y), free(T), free(tv);
}

int main(void)
{
    double *d, *e;
    /* degenerate orders */
    for (int64_t n = 0; n <= 2; ++n) {
        d = dalloc(n);
        e = dalloc(n - 1);
        for (int64_t i = 0; i < n; ++i) d[i] = (double)i;
        for (int64_t i = 0; i + 1 < n; ++i) e[i] = 0.5;
        run_path(n, d, e);
        free(d), free(e);
    }
    /* glued W21+: coincident eigenvalues and clusters of 2 and 4 members; zero glue splits */
    int64_t n = glued(2, 1e-10, &d, &e);
    run_path(n, d, e);
    free(d), free(e);
    n = glued(3, 0.0, &d, &e);
    run_path(n, d, e);
    free(d), free(e);
    /* uniform random, one matrix with exact zeros in e */
    n = 50;
    d = dalloc(n);
    e = dalloc(n - 1);
    uniform(n, 5, d, e);
    run_path(n, d, e);
    e[0] = e[20] = e[21] = e[n - 2] = 0.0;
    run_path(n, d, e);
    /* a diagonal T */
    for (int64_t i = 0; i + 1 < n; ++i) e[i] = 0.0;
    run_path(n, d, e);
    free(d), free(e);
    run_orth(30, 1);
    run_orth(30, 12);
    run_orth(12, 12);
    printf("ok\n");
    return 0;
}
