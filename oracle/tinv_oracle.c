/*
 * tinv_oracle.c -- plain, slow, single-threaded CPU FP64 oracle for inverse iteration with
 * MGS / Householder / compact-WY (CWY) reorthogonalization, written from
 * Ishigami, Kimura, Nakamura, arXiv:1209.1910.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the benchmark's
 * CPU-baseline leg, never by the product path.  It shares no code with the CUDA library.
 * Built with -ffp-contract=off so that every operation is rounded exactly as written.
 *
 * What each function follows:
 *   orc_start_value     -- random start vector (Alg. 1 / Alg. 4 "generate from random numbers"),
 *                          read as U[-1,1) from a counter-based SplitMix64 keyed by (seed, j).
 *   orc_bisect          -- eigenvalue approximations by bisection (Sec. 5.1, DSTEBZ's role).
 *   orc_plan            -- ||T||_1, the cluster tolerance 1e-3*||T|| and cluster heads j_1
 *                          (Sec. 2.1 Peters-Wilkinson test; Alg. 1 / Alg. 4), plus the
 *                          DSTEIN perturbation of coincident shifts.
 *   orc_lagtf/lagts     -- the shifted solve of Eq. 1 by LU with scaled partial pivoting.
 *   orc_orth_mgs        -- MGS (Alg. 1 inner loop, Sec. 2.2).
 *   orc_orth_house      -- Householder orthogonalization (Alg. 2, Eq. yt).
 *   orc_orth_cwy_*      -- compact-WY orthogonalization (Alg. 3) in the ordinary BLAS form
 *                          (Sec. 3.3.1) and the new form (Sec. 3.3.2), Eqs. cwy1/cwy2.
 *   orc_orth_cwy_block  -- compact WY over blocks of columns (Sec. 3.2, Eqs. cwy1/cwy2).
 *   orc_tinv            -- classical inverse iteration (Alg. 1) and DSTEIN-cWY (Alg. 4).
 *   orc_tinv_blocked    -- DSTEIN-cWY with a cluster's members orthogonalized in blocks.
 *   orc_jacobi          -- cyclic Jacobi (Golub & Van Loan), brute force for small n.
 *
 * Readings of points the paper leaves open:
 *   - q_j is formed with T_j, not T_j^T (Sec. 3.3.1/3.3.2 print T^T; Eq. cwy2 needs T).
 *   - the first q of Alg. 3 is formed with e_1 (printed e_j).
 *   - "Normalize v" before the solve is DSTEIN's 1-norm scaling
 *       v <- v * n*||T||_1*max(eps,|u_nn|) / ||v||_1.
 *   - "Until some condition": success when ||x||_inf >= sqrt(0.1/n); stop after EXTRA+1 = 3
 *     successes or MAXITS = 5 sweeps (DSTEIN's documented parameters).
 *   - After CWY the tested iterate is x = -c*q (q as printed, sign-flipped), which equals the
 *     MGS-orthogonalized iterate (I - Q Q^T) v; the next sweep starts from it.
 *   - Coincident shifts: if w_j - w'_{j-1} < 10*eps*|w_j| then w'_j = w'_{j-1} + 10*eps*|w_j|.
 *   - Tiny pivots in the solve (DLAGTS, job -1: U's diagonal is perturbed only to avoid
 *     overflow, by at least tol = eps*max|U|): u0_k is replaced by sign(u0_k)*tol, sign(0) = +,
 *     iff |u0_k| < DBL_MIN*max(1, |u1_k|, |u2_k|), i.e. iff a quotient of row k by u0_k could
 *     overflow; the decision depends on U alone, not on the right-hand side.
 *   - Breakdown (remainder exactly zero): CWY/Householder complete the basis with the first
 *     free unit vector (u_hat := e_1); MGS restarts from a fresh random vector. Either way
 *     the sweep does not count as a success.
 */
#include "tinv_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define EPS DBL_EPSILON
#define MAXITS 5
#define EXTRA 2
#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double sgn(double a) { return a < 0.0 ? -1.0 : 1.0; } /* sgn(0) = +1 */

/* ------------------------------------------------------------------------------------ */
/* Random start vectors                                                                  */
/* ------------------------------------------------------------------------------------ */

uint64_t orc_sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_sm64_next(uint64_t* state)
{
    *state += SM64_GAMMA;
    return orc_sm64_mix(*state);
}

double orc_start_value(uint64_t seed, int64_t j, int attempt, int64_t i)
{
    /* key = output number 8j+attempt+1 of SplitMix64 seeded with `seed`;
       value = output number i+1 of SplitMix64 seeded with `key`. */
    uint64_t key = orc_sm64_mix(seed + (uint64_t)(8 * j + attempt + 1) * SM64_GAMMA);
    uint64_t x = orc_sm64_mix(key + (uint64_t)(i + 1) * SM64_GAMMA);
    double u01 = (double)(x >> 11) * 0x1.0p-53; /* [0,1), exact */
    return 2.0 * u01 - 1.0;                      /* [-1,1), exact */
}

/* ------------------------------------------------------------------------------------ */
/* Norm, Sturm count, bisection                                                          */
/* ------------------------------------------------------------------------------------ */

double orc_onenorm(int64_t n, const double* d, const double* e)
{
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = fabs(d[i]);
        if (i > 0) s = s + fabs(e[i - 1]);
        if (i < n - 1) s = s + fabs(e[i]);
        if (s > nrm) nrm = s;
    }
    return nrm;
}

/* Unreduced blocks.  The paper takes its eigenvalues and their blocks from DSTEBZ and is silent
 * on the splitting rule; the reading taken here: the entry e_i is negligible, and row i ends a
 * block, iff |e_i| <= eps ||T||_1.  Dropping it changes T by at most eps ||T||_1 in norm, within
 * the residual bound the method already has.  isplit[b] = one past the last row of block b. */
int64_t orc_split(int64_t n, const double* d, const double* e, int64_t* isplit)
{
    if (n <= 0) return 0;
    double tol = EPS * orc_onenorm(n, d, e);
    int64_t nb = 0;
    for (int64_t i = 0; i < n - 1; ++i) {
        if (fabs(e[i]) <= tol) {
            isplit[nb] = i + 1;
            nb = nb + 1;
        }
    }
    isplit[nb] = n;
    return nb + 1;
}

int64_t orc_sturm_count(int64_t n, const double* d, const double* e, double x, double pivmin)
{
    int64_t cnt = 0;
    double q = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (i == 0)
            q = d[0] - x;
        else
            q = (d[i] - x) - (e[i - 1] * e[i - 1]) / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) cnt++;
    }
    return cnt;
}

void orc_bisect(int64_t n, const double* d, const double* e, double* w)
{
    if (n <= 0) return;
    double glo = INFINITY, ghi = -INFINITY, emax2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i < n - 1) {
            r += fabs(e[i]);
            emax2 = dmax(emax2, e[i] * e[i]);
        }
        glo = dmin(glo, d[i] - r);
        ghi = dmax(ghi, d[i] + r);
    }
    double pivmin = DBL_MIN * dmax(1.0, emax2);
    double bnd = dmax(fabs(glo), fabs(ghi));
    double widen = 2.0 * EPS * bnd * (double)n + 2.0 * pivmin;
    glo -= widen;
    ghi += widen;
    double onenrm = orc_onenorm(n, d, e);
    for (int64_t k = 0; k < n; ++k) {
        double lo = glo, hi = ghi;
        for (int it = 0; it < 4000; ++it) {
            double tol = dmax(2.0 * EPS * dmax(fabs(lo), fabs(hi)), EPS * onenrm);
            if (hi - lo <= tol) break;
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (orc_sturm_count(n, d, e, mid, pivmin) <= k)
                lo = mid;
            else
                hi = mid;
        }
        w[k] = 0.5 * (lo + hi);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Cluster plan (Sec. 2.1, Alg. 1, Alg. 4)                                              */
/* ------------------------------------------------------------------------------------ */

void orc_plan(int64_t n, const double* d, const double* e, int64_t m, const double* w,
              double* wp, int64_t* head, double* onenrm_out, double* ortol_out,
              double* dtpcrt_out)
{
    double onenrm = orc_onenorm(n, d, e);
    double ortol = 1e-3 * onenrm;
    double dtpcrt = sqrt(0.1 / (double)n);
    double xjm = 0.0;
    int64_t j1 = 0;
    for (int64_t j = 0; j < m; ++j) {
        double xj = w[j];
        if (j > 0) {
            double pertol = 10.0 * fabs(EPS * xj);
            if (xj - xjm < pertol) xj = xjm + pertol;
            if (fabs(xj - xjm) > ortol) j1 = j; /* gap > 1e-3*||T||: new cluster */
        } else {
            j1 = 0;
        }
        wp[j] = xj;
        head[j] = j1;
        xjm = xj;
    }
    if (onenrm_out) *onenrm_out = onenrm;
    if (ortol_out) *ortol_out = ortol;
    if (dtpcrt_out) *dtpcrt_out = dtpcrt;
}

/* ------------------------------------------------------------------------------------ */
/* Shifted tridiagonal LU and solve (Eq. 1)                                               */
/* ------------------------------------------------------------------------------------ */

/* Factor T - lambda*I = P L U.  U has diagonal u0[0..n), first superdiagonal u1[0..n-1),
 * second superdiagonal u2[0..n-1) (nonzero only where rows were interchanged).  L is unit
 * lower bidiagonal with multipliers l[0..n-1).  piv[k] = 1 iff rows k and k+1 were
 * interchanged at step k.  Row k+1 becomes the pivot row when its scaled subdiagonal entry
 * |c_k| / (|c_k| + |a_{k+1}| + |b_{k+1}|) exceeds the scaled pivot |a_k| / (|a_k| + |b_k|)
 * of the current row (a tie keeps the current row). */
void orc_lagtf(int64_t n, const double* d, const double* e, double lambda,
               double* u0, double* u1, double* u2, double* l, unsigned char* piv)
{
    if (n <= 0) return;
    double ak = d[0] - lambda;           /* diagonal of the current pivot row      */
    double bk = (n > 1) ? e[0] : 0.0;    /* superdiagonal of the current pivot row */
    for (int64_t k = 0; k + 1 < n; ++k) {
        double ck = e[k];                            /* entry below the pivot        */
        double a1 = d[k + 1] - lambda;               /* diagonal of row k+1          */
        double b1 = (k + 2 < n) ? e[k + 1] : 0.0;    /* superdiagonal of row k+1     */
        double scale1 = fabs(ak) + fabs(bk);
        double scale2 = (fabs(ck) + fabs(a1)) + fabs(b1);
        double piv1 = (ak == 0.0) ? 0.0 : fabs(ak) / scale1;
        double piv2 = (ck == 0.0) ? 0.0 : fabs(ck) / scale2;
        if (piv2 <= piv1) {
            double lk = (ck == 0.0) ? 0.0 : ck / ak;
            u0[k] = ak;
            u1[k] = bk;
            u2[k] = 0.0;
            l[k] = lk;
            piv[k] = 0;
            ak = a1 - lk * bk;
            bk = b1;
        } else {
            double lk = ak / ck;
            u0[k] = ck;
            u1[k] = a1;
            u2[k] = b1;
            l[k] = lk;
            piv[k] = 1;
            ak = bk - lk * a1;
            bk = -(lk * b1);
        }
    }
    u0[n - 1] = ak;
}

/* Solve with the factors of orc_lagtf: first P and L, then U by back substitution.  A
 * diagonal entry of U so small that a quotient of its row by it could overflow,
 * |u0_k| < DBL_MIN*max(1, |u1_k|, |u2_k|) (zero included), is replaced by sign(u0_k)*tol with
 * tol = eps*max|U| (sign(0) = +), the minimum perturbation of DLAGTS's job -1.  Returns tol. */
double orc_lagts(int64_t n, const double* u0, const double* u1, const double* u2,
                 const double* l, const unsigned char* piv, double* y)
{
    if (n <= 0) return EPS;
    double umax = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        umax = dmax(umax, fabs(u0[k]));
        if (k + 1 < n) umax = dmax(umax, fabs(u1[k]));
        if (k + 1 < n) umax = dmax(umax, fabs(u2[k]));
    }
    double tol = EPS * umax;
    if (tol == 0.0) tol = EPS;
    for (int64_t k = 0; k + 1 < n; ++k) {
        if (piv[k]) {
            double tmp = y[k];
            y[k] = y[k + 1];
            y[k + 1] = tmp - l[k] * y[k];
        } else {
            y[k + 1] = y[k + 1] - l[k] * y[k];
        }
    }
    for (int64_t k = n - 1; k >= 0; --k) {
        double temp = y[k];
        if (k + 1 < n) temp = temp - u1[k] * y[k + 1];
        if (k + 2 < n) temp = temp - u2[k] * y[k + 2];
        double ak = u0[k];
        double big = 1.0;
        if (k + 1 < n) big = dmax(big, fabs(u1[k]));
        if (k + 1 < n) big = dmax(big, fabs(u2[k]));
        if (fabs(ak) < DBL_MIN * big) ak = (ak >= 0.0) ? tol : -tol;
        y[k] = temp / ak;
    }
    return tol;
}

/* ------------------------------------------------------------------------------------ */
/* Small dense helpers (plain loops)                                                     */
/* ------------------------------------------------------------------------------------ */

static double dot(int64_t n, const double* x, const double* y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

static double nrm2(int64_t n, const double* x)
{
    /* plain definition; inputs here are O(1) after scaling, so no overflow guard needed */
    return sqrt(dot(n, x, x));
}

/* ------------------------------------------------------------------------------------ */
/* Householder reflector (Sec. 3.1, Eq. yt)                                                */
/* ------------------------------------------------------------------------------------ */

/* Given u_hat = u[j..n) (length len), build y_hat = [u_jj - c, u_{j+1..n}] and return c;
 * c = -sgn(u_jj) * ||u_hat||.  On an exactly zero u_hat the remainder is replaced by the
 * first free unit vector (breakdown; *broke = 1). */
static double reflector(int64_t len, const double* uhat, double* yhat, int* broke)
{
    double nrm = nrm2(len, uhat);
    *broke = 0;
    if (!(nrm > 0.0) || !isfinite(nrm)) {
        *broke = 1;
        for (int64_t i = 0; i < len; ++i) yhat[i] = 0.0;
        /* u_hat := e_1: c = -1, y_hat = e_1 - c e_1 = 2 e_1 */
        yhat[0] = 2.0;
        return -1.0;
    }
    double c = -sgn(uhat[0]) * nrm;
    for (int64_t i = 0; i < len; ++i) yhat[i] = uhat[i];
    yhat[0] = uhat[0] - c;
    return c;
}

/* ------------------------------------------------------------------------------------ */
/* Stand-alone orthogonalizers (Sec. 3)                                                    */
/* ------------------------------------------------------------------------------------ */

/* MGS: q_j = normalize(v_j - sum_i <., q_i> q_i), projections applied one at a time. */
double orc_orth_mgs(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q, int64_t ldq)
{
    int64_t nfma = 0; /* multiply-adds executed (Table 1 accounting) */
    for (int64_t j = 0; j < m; ++j) {
        double* q = Q + j * ldq;
        for (int64_t r = 0; r < n; ++r) q[r] = V[r + j * ldv];
        for (int64_t i = 0; i < j; ++i) {
            const double* qi = Q + i * ldq;
            double h = 0.0;
            for (int64_t r = 0; r < n; ++r) { h += q[r] * qi[r]; nfma++; }
            for (int64_t r = 0; r < n; ++r) { q[r] = q[r] - h * qi[r]; nfma++; }
        }
        double nr = nrm2(n, q);
        for (int64_t r = 0; r < n; ++r) q[r] = q[r] / nr;
    }
    return 2.0 * (double)nfma;
}

/* Apply H_i = I - t_i y_i y_i^T (y_i zero above row i) to x in place; returns the number
 * of multiply-adds executed. */
static int64_t apply_reflector(int64_t n, int64_t i, const double* yi, double ti, double* x)
{
    double s = 0.0;
    for (int64_t r = i; r < n; ++r) s += yi[r] * x[r];
    s = ti * s;
    for (int64_t r = i; r < n; ++r) x[r] = x[r] - s * yi[r];
    return 2 * (n - i);
}

/* Alg. 2: u_j = H_{j-1}...H_1 v_j; y_j, t_j from u_j (Eq. yt, t = 2/||y||^2);
 * q_j = H_1...H_j e_j.  Y (n x m) and tv (m) receive the reflectors. */
double orc_orth_house(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q, int64_t ldq,
                      double* Y, double* tv)
{
    int64_t nfma = 0;
    double* Yw = Y ? Y : (double*)calloc((size_t)(n * m), sizeof(double));
    double* tw = tv ? tv : (double*)calloc((size_t)m, sizeof(double));
    double* u = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < m; ++j) {
        for (int64_t r = 0; r < n; ++r) u[r] = V[r + j * ldv];
        for (int64_t i = 0; i < j; ++i) nfma += apply_reflector(n, i, Yw + i * n, tw[i], u);
        double* yj = Yw + j * n;
        for (int64_t r = 0; r < j; ++r) yj[r] = 0.0;
        int broke;
        reflector(n - j, u + j, yj + j, &broke);
        double yy = dot(n - j, yj + j, yj + j);
        tw[j] = 2.0 / yy;
        double* q = Q + j * ldq;
        for (int64_t r = 0; r < n; ++r) q[r] = 0.0;
        q[j] = 1.0;
        for (int64_t i = j; i >= 0; --i) nfma += apply_reflector(n, i, Yw + i * n, tw[i], q);
    }
    free(u);
    if (!Y) free(Yw);
    if (!tv) free(tw);
    return 2.0 * (double)nfma;
}

/* Alg. 3 in the ordinary BLAS form of Sec. 3.3.1:
 *   u_j = v_j - Y_{j-1} T_{j-1}^T Y_{j-1}^T v_j  (DCOPY, DGEMV, DTRMV, DGEMV)
 *   y_j, t_j = 2/||y_j||^2                        (Eq. yt)
 *   t_hat = -t_j T_{j-1} Y_{j-1}^T y_j            (DGEMV, DTRMV)
 *   q_j = e_j - Y_j T_j Y_j^T e_j                 (Y_j^T e_j = row j of Y_j; T_j, reading c1)
 * Y is n x m (full columns, zeros above the diagonal), T is m x m upper triangular. */
double orc_orth_cwy_ordinary(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q,
                             int64_t ldq, double* Y, double* T)
{
    int64_t nfma = 0;
    double* Yw = Y ? Y : (double*)calloc((size_t)(n * m), sizeof(double));
    double* Tw = T ? T : (double*)calloc((size_t)(m * m), sizeof(double));
    double* u = (double*)malloc(sizeof(double) * (size_t)n);
    double* s = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double* s2 = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    for (int64_t j = 0; j < m; ++j) {
        /* line 5: u_j = (I - Y T^T Y^T) v_j over full columns of Y */
        for (int64_t r = 0; r < n; ++r) u[r] = V[r + j * ldv];
        for (int64_t i = 0; i < j; ++i) {
            double acc = 0.0;
            for (int64_t r = 0; r < n; ++r) { acc += Yw[r + i * n] * u[r]; nfma++; }
            s[i] = acc;
        }
        for (int64_t i = 0; i < j; ++i) { /* s2 = T^T s */
            double acc = 0.0;
            for (int64_t l2 = 0; l2 <= i; ++l2) { acc += Tw[l2 + i * m] * s[l2]; nfma++; }
            s2[i] = acc;
        }
        for (int64_t r = 0; r < n; ++r) {
            double acc = 0.0;
            for (int64_t i = 0; i < j; ++i) { acc += Yw[r + i * n] * s2[i]; nfma++; }
            u[r] = u[r] - acc;
        }
        /* line 6: y_j and t_j from u_j */
        double* yj = Yw + j * n;
        for (int64_t r = 0; r < j; ++r) yj[r] = 0.0;
        int broke;
        reflector(n - j, u + j, yj + j, &broke);
        double tj = 2.0 / dot(n, yj, yj);
        /* line 7: t_hat = -t_j T_{j-1} Y_{j-1}^T y_j */
        for (int64_t i = 0; i < j; ++i) {
            double acc = 0.0;
            for (int64_t r = 0; r < n; ++r) { acc += Yw[r + i * n] * yj[r]; nfma++; }
            s[i] = acc;
        }
        for (int64_t i = 0; i < j; ++i) {
            double acc = 0.0;
            for (int64_t l2 = i; l2 < j; ++l2) { acc += Tw[i + l2 * m] * s[l2]; nfma++; }
            Tw[i + j * m] = -tj * acc;
        }
        for (int64_t i = j + 1; i < m; ++i) Tw[i + j * m] = 0.0;
        Tw[j + j * m] = tj;
        /* line 8: q_j = e_j - Y_j T_j (Y_j^T e_j) */
        for (int64_t i = 0; i <= j; ++i) s[i] = Yw[j + i * n];
        for (int64_t i = 0; i <= j; ++i) {
            double acc = 0.0;
            for (int64_t l2 = i; l2 <= j; ++l2) { acc += Tw[i + l2 * m] * s[l2]; nfma++; }
            s2[i] = acc;
        }
        double* q = Q + j * ldq;
        for (int64_t r = 0; r < n; ++r) {
            double acc = 0.0;
            for (int64_t i = 0; i <= j; ++i) { acc += Yw[r + i * n] * s2[i]; nfma++; }
            q[r] = (r == j ? 1.0 : 0.0) - acc;
        }
    }
    free(u);
    free(s);
    free(s2);
    if (!Y) free(Yw);
    if (!T) free(Tw);
    return 2.0 * (double)nfma;
}

/* One step of the new CWY implementation (Sec. 3.3.2) for column k (0-based; k previous
 * reflectors in Y[:,0..k), T[0..k,0..k)).  Input v (length n).  On return Y[:,k], T[:,k]
 * hold the new reflector, q (length n) holds the sign-flipped q = (Y T Y^T - I) e_k, and the
 * return value is c.  ld of Y is n, of T is ldt.  *broke flags a zero remainder. */
static double cwy_new_step(int64_t n, int64_t k, double* Y, double* T, int64_t ldt,
                           const double* v, double* q, double* work, int* broke, double* flops)
{
    int64_t nfma = 0;          /* multiply-adds executed (Table 1 accounting) */
    double* s = work;          /* k   */
    double* uh = work + n + 1; /* n-k */
    /* s = L_k^T v_check + Yhat_k^T v_hat  (DTRMV + DGEMV) */
    for (int64_t i = 0; i < k; ++i) {
        double acc = 0.0;
        for (int64_t r = i; r < k; ++r) { acc += Y[r + i * n] * v[r]; nfma++; } /* L_k^T v_check */
        double acc2 = 0.0;
        for (int64_t r = k; r < n; ++r) { acc2 += Y[r + i * n] * v[r]; nfma++; } /* Yhat^T v_hat */
        s[i] = acc + acc2;
    }
    /* s <- T_k^T s (DTRMV), computed from the bottom so each s[i] uses the old s[0..i] */
    for (int64_t i = k - 1; i >= 0; --i) {
        double acc = 0.0;
        for (int64_t l2 = 0; l2 <= i; ++l2) { acc += T[l2 + i * ldt] * s[l2]; nfma++; }
        s[i] = acc;
    }
    /* u_hat = v_hat - Yhat_k s (DCOPY + DGEMV) */
    for (int64_t r = k; r < n; ++r) {
        double acc = 0.0;
        for (int64_t i = 0; i < k; ++i) { acc += Y[r + i * n] * s[i]; nfma++; }
        uh[r - k] = v[r] - acc;
    }
    /* y_k, c_k (DNRM2) and t_k = 1/(c^2 - u_kk c) */
    double* yk = Y + k * n;
    for (int64_t r = 0; r < k; ++r) yk[r] = 0.0;
    double c = reflector(n - k, uh, yk + k, broke);
    double ukk = *broke ? 1.0 : uh[0];
    double tk = 1.0 / (c * c - ukk * c);
    /* t_hat = -t_k T_k (Yhat_k^T y_hat)  (DGEMV + DTRMV; the L part meets zeros) */
    double* g = work; /* reuse: s is no longer needed */
    for (int64_t i = 0; i < k; ++i) {
        double acc = 0.0;
        for (int64_t r = k; r < n; ++r) { acc += Y[r + i * n] * yk[r]; nfma++; }
        g[i] = -tk * acc;
    }
    for (int64_t i = 0; i < k; ++i) {
        double acc = 0.0;
        for (int64_t l2 = i; l2 < k; ++l2) { acc += T[i + l2 * ldt] * g[l2]; nfma++; }
        T[i + k * ldt] = acc;
    }
    T[k + k * ldt] = tk;
    /* q = (Y_{k+1} T_{k+1} Y_{k+1}^T - I) e_k:
       x = T_{k+1} (row k of Y_{k+1}) (DCOPY + DTRMV with T, reading c1),
       q_check = L_{k+1} x (DTRMV), q_hat = Yhat_{k+1} x (DGEMV), q_kk -= 1. */
    double* x = work;
    for (int64_t i = 0; i <= k; ++i) x[i] = Y[k + i * n];
    for (int64_t i = 0; i <= k; ++i) {
        double acc = 0.0;
        for (int64_t l2 = i; l2 <= k; ++l2) { acc += T[i + l2 * ldt] * x[l2]; nfma++; }
        x[i] = acc; /* x[l2] for l2 > i still holds the old row entries */
    }
    for (int64_t r = 0; r <= k; ++r) {
        double acc = 0.0;
        for (int64_t i = 0; i <= r; ++i) { acc += Y[r + i * n] * x[i]; nfma++; }
        q[r] = acc;
    }
    for (int64_t r = k + 1; r < n; ++r) {
        double acc = 0.0;
        for (int64_t i = 0; i <= k; ++i) { acc += Y[r + i * n] * x[i]; nfma++; }
        q[r] = acc;
    }
    q[k] = q[k] - 1.0;
    if (flops) *flops += 2.0 * (double)nfma;
    return c;
}

/* Alg. 3 with the new implementation of Sec. 3.3.2 (Q gets the sign-flipped q_j). */
double orc_orth_cwy_new(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q,
                        int64_t ldq, double* Y, double* T)
{
    double flops = 0.0;
    double* Yw = Y ? Y : (double*)calloc((size_t)(n * m), sizeof(double));
    double* Tw = T ? T : (double*)calloc((size_t)(m * m), sizeof(double));
    double* work = (double*)malloc(sizeof(double) * (size_t)(2 * n + 2));
    for (int64_t j = 0; j < m; ++j) {
        int broke;
        for (int64_t i = j + 1; i < m; ++i) Tw[i + j * m] = 0.0;
        cwy_new_step(n, j, Yw, Tw, m, V + j * ldv, Q + j * ldq, work, &broke, &flops);
    }
    free(work);
    if (!Y) free(Yw);
    if (!T) free(Tw);
    return flops;
}

/* ------------------------------------------------------------------------------------ */
/* Compact WY over a block of columns (Sec. 3.2, Eqs. cwy1 and cwy2)                       */
/* ------------------------------------------------------------------------------------ */

/* One block step: the columns W (n x bb, ld n) are orthogonalized against the k0 reflectors
 * in Y[:, 0..k0), T[0..k0, 0..k0) and among themselves, and their reflectors are appended as
 * columns k0 .. k0+bb-1 of Y and T (ld n and ldt):
 *   (1) W <- Q_k0^T W = W - Y T^T (Y^T W)                  (Q_k0 = I - Y T Y^T, Eq. cwy2)
 *   (2) Householder QR of the rows k0.. of W, one column at a time (Alg. 2 on the panel):
 *       column c gives y (Eq. yt, zero above row k0+c), c_c = -sgn(u_1) ||u_hat|| and
 *       t_c = 1/(c_c^2 - u_1 c_c); H_c = I - t_c y y^T is applied to the later columns; T
 *       grows by the recurrence of Eq. cwy1: T[0..col, col] = -t_c T (Y^T y), T[col, col] = t_c.
 *   (3) Q[:, c] = (Y T Y^T - I) e_{k0+c} with the reflectors 0..k0+c (the sign-flipped q of
 *       Sec. 3.3.2; later reflectors leave e_{k0+c} unchanged).
 * cvals[c] receives c_c and broke[c] = 1 where the remainder was exactly zero (it is then
 * replaced by the first free unit vector, as in the one-column step).  Returns the flops. */
static double cwy_block_step(int64_t n, int64_t k0, int64_t bb, double* Y, double* T, int64_t ldt,
                             double* W, double* Q, int64_t ldq, double* cvals, int* broke,
                             double* work)
{
    int64_t nfma = 0;
    double* s = work;              /* k0 + bb */
    double* s2 = work + (n + 1);   /* k0 + bb */
    /* (1) W <- W - Y_k0 T_k0^T (Y_k0^T W), one column at a time */
    for (int64_t c = 0; c < bb; ++c) {
        double* wc = W + c * n;
        for (int64_t i = 0; i < k0; ++i) {
            double acc = 0.0;
            for (int64_t r = i; r < n; ++r) { acc += Y[r + i * n] * wc[r]; nfma++; }
            s[i] = acc;
        }
        for (int64_t i = 0; i < k0; ++i) { /* s2 = T^T s */
            double acc = 0.0;
            for (int64_t l2 = 0; l2 <= i; ++l2) { acc += T[l2 + i * ldt] * s[l2]; nfma++; }
            s2[i] = acc;
        }
        for (int64_t r = 0; r < n; ++r) {
            double acc = 0.0;
            int64_t top = r < k0 ? r + 1 : k0;
            for (int64_t i = 0; i < top; ++i) { acc += Y[r + i * n] * s2[i]; nfma++; }
            wc[r] = wc[r] - acc;
        }
    }
    /* (2) Householder QR of the panel rows k0.., T by Eq. cwy1 */
    for (int64_t c = 0; c < bb; ++c) {
        const int64_t col = k0 + c;
        double* yk = Y + col * n;
        for (int64_t r = 0; r < col; ++r) yk[r] = 0.0;
        cvals[c] = reflector(n - col, W + c * n + col, yk + col, &broke[c]);
        const double u1 = broke[c] ? 1.0 : W[col + c * n];
        const double tc = 1.0 / (cvals[c] * cvals[c] - u1 * cvals[c]);
        for (int64_t c2 = c + 1; c2 < bb; ++c2) { /* H_c on the later columns */
            double* w2 = W + c2 * n;
            double acc = 0.0;
            for (int64_t r = col; r < n; ++r) { acc += yk[r] * w2[r]; nfma++; }
            acc = tc * acc;
            for (int64_t r = col; r < n; ++r) { w2[r] = w2[r] - acc * yk[r]; nfma++; }
        }
        for (int64_t i = 0; i < col; ++i) { /* g = Y^T y over the rows where y is nonzero */
            double acc = 0.0;
            for (int64_t r = col; r < n; ++r) { acc += Y[r + i * n] * yk[r]; nfma++; }
            s[i] = -tc * acc;
        }
        for (int64_t i = 0; i < col; ++i) {
            double acc = 0.0;
            for (int64_t l2 = i; l2 < col; ++l2) { acc += T[i + l2 * ldt] * s[l2]; nfma++; }
            T[i + col * ldt] = acc;
        }
        for (int64_t i = col + 1; i < ldt; ++i) T[i + col * ldt] = 0.0;
        T[col + col * ldt] = tc;
    }
    /* (3) Q[:, c] = (Y T Y^T - I) e_col with the reflectors 0..col */
    for (int64_t c = 0; c < bb; ++c) {
        const int64_t col = k0 + c;
        double* q = Q + c * ldq;
        for (int64_t i = 0; i <= col; ++i) s[i] = Y[col + i * n];
        for (int64_t i = 0; i <= col; ++i) {
            double acc = 0.0;
            for (int64_t l2 = i; l2 <= col; ++l2) { acc += T[i + l2 * ldt] * s[l2]; nfma++; }
            s2[i] = acc;
        }
        for (int64_t r = 0; r < n; ++r) {
            double acc = 0.0;
            int64_t top = r < col ? r + 1 : col + 1;
            for (int64_t i = 0; i < top; ++i) { acc += Y[r + i * n] * s2[i]; nfma++; }
            q[r] = acc - (r == col ? 1.0 : 0.0);
        }
    }
    return 2.0 * (double)nfma;
}

/* Alg. 3 with the columns taken nb at a time through cwy_block_step (Q: sign-flipped q_j). */
double orc_orth_cwy_block(int64_t n, int64_t m, const double* V, int64_t ldv, int64_t nb,
                          double* Q, int64_t ldq, double* Y, double* T)
{
    double flops = 0.0;
    if (nb < 1) nb = 1;
    double* Yw = Y ? Y : (double*)calloc((size_t)(n * m), sizeof(double));
    double* Tw = T ? T : (double*)calloc((size_t)(m * m), sizeof(double));
    double* W = (double*)malloc(sizeof(double) * (size_t)(n * nb));
    double* work = (double*)malloc(sizeof(double) * (size_t)(2 * n + 2 * m + 4));
    double* cv = (double*)malloc(sizeof(double) * (size_t)nb);
    int* br = (int*)malloc(sizeof(int) * (size_t)nb);
    for (int64_t k0 = 0; k0 < m; k0 += nb) {
        const int64_t bb = (m - k0 < nb) ? m - k0 : nb;
        for (int64_t c = 0; c < bb; ++c)
            for (int64_t r = 0; r < n; ++r) W[r + c * n] = V[r + (k0 + c) * ldv];
        flops += cwy_block_step(n, k0, bb, Yw, Tw, m, W, Q + k0 * ldq, ldq, cv, br, work);
    }
    free(W);
    free(work);
    free(cv);
    free(br);
    if (!Y) free(Yw);
    if (!T) free(Tw);
    return flops;
}

/* Inverse iteration with blocked compact-WY reorthogonalization.  Heads and singletons are as
 * in orc_tinv.  After a cluster's head, its other mc-1 members are split into nblk =
 * ceil((mc-1)/nb) blocks, block b holding the members 1 + b + nblk c (evenly spread over the
 * cluster), processed b = 0, 1, ...; the reflectors are appended to Y and T in that order.
 * Every member of a block keeps its own shift, LU and start vector (the keys of orc_tinv), and
 * the block sweeps together: each member's iterate is scaled and solved (Eq. 1), then the block
 * is orthogonalized by cwy_block_step against the reflectors of the blocks before it and among
 * itself, in member order.  Member c's tested iterate is x_c = -c_c q_c (the
 * orthogonalized iterate, as in orc_tinv's CWY path); a success is ||x_c||_inf >= dtpcrt
 * without breakdown.  The block stops when every member has EXTRA+1 successes or after MAXITS
 * sweeps; each sweep recomputes the block's columns of Y and T.  A member without EXTRA+1
 * successes is counted as not converged.  nb = 1 is orc_tinv's CWY iteration. */
int64_t orc_tinv_blocked(int64_t n, const double* d, const double* e, int64_t m, const double* w,
                         int64_t j0, double* Z, int64_t ldz, int64_t nb, uint64_t seed,
                         int64_t* ifail, int32_t* iters, orc_stats* st)
{
    if (n <= 0 || m <= 0) return 0;
    if (nb < 1) nb = 1;
    if (n == 1) {
        for (int64_t j = 0; j < m; ++j) {
            Z[j * ldz] = 1.0;
            if (iters) iters[j] = 0;
        }
        return 0;
    }
    double* wp = (double*)malloc(sizeof(double) * (size_t)m);
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    double onenrm, ortol, dtpcrt;
    orc_plan(n, d, e, m, w, wp, head, &onenrm, &ortol, &dtpcrt);
    int64_t mcmax = 1;
    for (int64_t j = 0, cnt = 0; j < m; ++j) {
        cnt = (head[j] == j) ? 1 : cnt + 1;
        if (cnt > mcmax) mcmax = cnt;
    }
    /* factors of every member of a block */
    double* u0 = (double*)malloc(sizeof(double) * (size_t)(n * nb));
    double* u1 = (double*)malloc(sizeof(double) * (size_t)(n * nb));
    double* u2 = (double*)malloc(sizeof(double) * (size_t)(n * nb));
    double* l = (double*)malloc(sizeof(double) * (size_t)(n * nb));
    unsigned char* piv = (unsigned char*)malloc((size_t)(n * nb));
    double* unn = (double*)malloc(sizeof(double) * (size_t)nb);
    double* W = (double*)malloc(sizeof(double) * (size_t)(n * nb));  /* iterates / panel */
    double* Qb = (double*)malloc(sizeof(double) * (size_t)(n * nb)); /* sign-flipped q's */
    double* X = (double*)malloc(sizeof(double) * (size_t)(n * nb));  /* tested iterates */
    double* cv = (double*)malloc(sizeof(double) * (size_t)nb);
    int* br = (int*)malloc(sizeof(int) * (size_t)nb);
    int* nrmchk = (int*)malloc(sizeof(int) * (size_t)nb);
    double* work = (double*)malloc(sizeof(double) * (size_t)(2 * n + 2 * mcmax + 4));
    double* Y = (double*)calloc((size_t)(n * mcmax), sizeof(double));
    double* T = (double*)calloc((size_t)(mcmax * mcmax), sizeof(double));

    int64_t info = 0;
    for (int64_t j1 = 0; j1 < m;) {
        int64_t mc = 1;
        while (j1 + mc < m && head[j1 + mc] == j1) mc++;
        /* the head (or a singleton): inverse iteration without reorthogonalization */
        {
            double* v = X;
            orc_lagtf(n, d, e, wp[j1], u0, u1, u2, l, piv);
            const double un = fabs(u0[n - 1]);
            for (int64_t r = 0; r < n; ++r) v[r] = orc_start_value(seed, j0 + j1, 0, r);
            int cnt = 0, its = 0, conv = 0;
            while (its < MAXITS) {
                its++;
                double asum = 0.0;
                for (int64_t r = 0; r < n; ++r) asum += fabs(v[r]);
                double scl = (double)n * onenrm * dmax(EPS, un) / asum;
                for (int64_t r = 0; r < n; ++r) v[r] = scl * v[r];
                orc_lagts(n, u0, u1, u2, l, piv, v);
                double nrm = 0.0;
                for (int64_t r = 0; r < n; ++r) nrm = dmax(nrm, fabs(v[r]));
                if (nrm >= dtpcrt && ++cnt >= EXTRA + 1) {
                    conv = 1;
                    break;
                }
            }
            if (st) st->sweeps += its;
            if (iters) iters[j1] = its;
            if (!conv) {
                if (ifail) ifail[info] = j1;
                info++;
            }
            double nr = nrm2(n, v);
            int64_t jmax = 0;
            for (int64_t r = 1; r < n; ++r)
                if (fabs(v[r]) > fabs(v[jmax])) jmax = r;
            double sc = 1.0 / nr;
            if (v[jmax] < 0.0) sc = -sc;
            for (int64_t r = 0; r < n; ++r) Z[r + j1 * ldz] = sc * v[r];
        }
        if (mc > 1) {
            /* Alg. 4: Y_1 = [y_1], T_1 = [t_1] from the (final) head vector */
            const double* zh = Z + j1 * ldz;
            int broke;
            double c = reflector(n, zh, Y, &broke);
            double uh = broke ? 1.0 : zh[0];
            T[0] = 1.0 / (c * c - uh * c);
        }
        /* the members 1..mc-1 go to nblk blocks of at most nb, block b holding the members
           1 + b + nblk*c: the members that sweep together are spread evenly over the cluster,
           so near neighbours in the spectrum are orthogonalized against finished vectors */
        const int64_t nblk = (mc - 1 + nb - 1) / nb;
        int64_t kpos = 1;
        for (int64_t bi = 0; bi < nblk; ++bi) {
            const int64_t k0 = kpos; /* Y and T columns of this block: k0 .. k0+bb-1 */
            const int64_t bb = (mc - 1 - bi + nblk - 1) / nblk;
            kpos += bb;
            for (int64_t c = 0; c < bb; ++c) {
                const int64_t j = j1 + 1 + bi + nblk * c;
                orc_lagtf(n, d, e, wp[j], u0 + c * n, u1 + c * n, u2 + c * n, l + c * n, piv + c * n);
                unn[c] = fabs(u0[c * n + n - 1]);
                for (int64_t r = 0; r < n; ++r) X[r + c * n] = orc_start_value(seed, j0 + j, 0, r);
                nrmchk[c] = 0;
            }
            int its = 0, all = 0;
            while (its < MAXITS) {
                its++;
                for (int64_t c = 0; c < bb; ++c) {
                    double* v = X + c * n;
                    double asum = 0.0;
                    for (int64_t r = 0; r < n; ++r) asum += fabs(v[r]);
                    double scl = (double)n * onenrm * dmax(EPS, unn[c]) / asum;
                    for (int64_t r = 0; r < n; ++r) W[r + c * n] = scl * v[r];
                    orc_lagts(n, u0 + c * n, u1 + c * n, u2 + c * n, l + c * n, piv + c * n, W + c * n);
                }
                double fl = cwy_block_step(n, k0, bb, Y, T, mcmax, W, Qb, n, cv, br, work);
                if (st) st->orth_flops += fl;
                all = 1;
                for (int64_t c = 0; c < bb; ++c) {
                    double* x = X + c * n;
                    double nrm = 0.0;
                    for (int64_t r = 0; r < n; ++r) {
                        x[r] = -cv[c] * Qb[r + c * n];
                        nrm = dmax(nrm, fabs(x[r]));
                    }
                    if (br[c]) {
                        if (st) st->breakdowns++;
                    } else if (nrm >= dtpcrt) {
                        nrmchk[c]++;
                    }
                    if (nrmchk[c] < EXTRA + 1) all = 0;
                }
                if (all) break;
            }
            for (int64_t c = 0; c < bb; ++c) {
                const int64_t j = j1 + 1 + bi + nblk * c;
                const double* x = X + c * n;
                if (st) st->sweeps += its;
                if (iters) iters[j] = its;
                if (nrmchk[c] < EXTRA + 1) {
                    if (ifail) ifail[info] = j;
                    info++;
                }
                double nr = nrm2(n, x);
                int64_t jmax = 0;
                for (int64_t r = 1; r < n; ++r)
                    if (fabs(x[r]) > fabs(x[jmax])) jmax = r;
                double sc = 1.0 / nr;
                if (x[jmax] < 0.0) sc = -sc;
                for (int64_t r = 0; r < n; ++r) Z[r + j * ldz] = sc * x[r];
            }
        }
        j1 += mc;
    }
    free(wp);
    free(head);
    free(u0);
    free(u1);
    free(u2);
    free(l);
    free(piv);
    free(unn);
    free(W);
    free(Qb);
    free(X);
    free(cv);
    free(br);
    free(nrmchk);
    free(work);
    free(Y);
    free(T);
    return info;
}

/* ------------------------------------------------------------------------------------ */
/* Inverse iteration: Alg. 1 (MGS), Alg. 4 (CWY), Alg. 2 incrementally (HOUSE)             */
/* ------------------------------------------------------------------------------------ */

int64_t orc_tinv(int64_t n, const double* d, const double* e, int64_t m, const double* w,
                 int64_t j0, double* Z, int64_t ldz, int method, uint64_t seed,
                 int64_t* ifail, int32_t* iters, orc_stats* st)
{
    if (n <= 0 || m <= 0) return 0;
    if (n == 1) {
        for (int64_t j = 0; j < m; ++j) {
            Z[j * ldz] = 1.0;
            if (iters) iters[j] = 0;
        }
        return 0;
    }
    double* wp = (double*)malloc(sizeof(double) * (size_t)m);
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    double onenrm, ortol, dtpcrt;
    orc_plan(n, d, e, m, w, wp, head, &onenrm, &ortol, &dtpcrt);

    double* u0 = (double*)malloc(sizeof(double) * (size_t)n);
    double* u1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* u2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* l = (double*)malloc(sizeof(double) * (size_t)n);
    unsigned char* piv = (unsigned char*)malloc((size_t)n);
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    double* work = (double*)malloc(sizeof(double) * (size_t)(2 * n + 2));
    /* compact-WY state of the current cluster: Y (n x mc), T (mc x mc); sized for the largest
       cluster. HOUSE keeps Y and the scalars t_i in tv. */
    int64_t mcmax = 1;
    for (int64_t j = 0, cnt = 0; j < m; ++j) {
        cnt = (head[j] == j) ? 1 : cnt + 1;
        if (cnt > mcmax) mcmax = cnt;
    }
    double* Y = NULL;
    double* T = NULL;
    double* tv = NULL;
    if (method != ORC_MGS) {
        Y = (double*)calloc((size_t)(n * mcmax), sizeof(double));
        T = (double*)calloc((size_t)(mcmax * mcmax), sizeof(double));
        tv = (double*)calloc((size_t)mcmax, sizeof(double));
    }

    int64_t info = 0;
    for (int64_t j = 0; j < m; ++j) {
        int64_t j1 = head[j];
        int64_t jc = j - j1; /* position inside the cluster (Alg. 4) */
        double xj = wp[j];
        orc_lagtf(n, d, e, xj, u0, u1, u2, l, piv);
        double unn = fabs(u0[n - 1]);
        int attempt = 0;
        for (int64_t r = 0; r < n; ++r) v[r] = orc_start_value(seed, j0 + j, attempt, r);

        if (jc == 1 && method != ORC_MGS) {
            /* Alg. 4: Y_1 = [y_1], T_1 = [t_1] from the (final) head vector */
            const double* zh = Z + j1 * ldz;
            int broke;
            double c = reflector(n, zh, Y, &broke);
            double u11 = broke ? 1.0 : zh[0];
            double t1 = 1.0 / (c * c - u11 * c);
            T[0] = t1;
            tv[0] = 2.0 / dot(n, Y, Y);
        }

        int nrmchk = 0, its = 0, converged = 0;
        while (its < MAXITS) {
            its++;
            /* "Normalize": DSTEIN 1-norm scaling before the solve */
            double asum = 0.0;
            for (int64_t r = 0; r < n; ++r) asum += fabs(v[r]);
            double scl = (double)n * onenrm * dmax(EPS, unn) / asum;
            for (int64_t r = 0; r < n; ++r) v[r] = scl * v[r];
            /* Eq. 1 */
            orc_lagts(n, u0, u1, u2, l, piv, v);
            int success_allowed = 1;
            if (jc > 0) {
                if (method == ORC_MGS) {
                    /* Alg. 1: MGS against the previous members of the cluster */
                    for (int64_t i = j1; i < j; ++i) {
                        const double* zi = Z + i * ldz;
                        double h = dot(n, v, zi);
                        for (int64_t r = 0; r < n; ++r) v[r] = v[r] - h * zi[r];
                    }
                    if (st) st->orth_flops += 4.0 * (double)n * (double)jc;
                    double a2 = 0.0;
                    for (int64_t r = 0; r < n; ++r) a2 += fabs(v[r]);
                    if (!(a2 > 0.0)) { /* breakdown: restart from a fresh random vector */
                        attempt++;
                        for (int64_t r = 0; r < n; ++r)
                            v[r] = orc_start_value(seed, j0 + j, attempt, r);
                        success_allowed = 0;
                        if (st) st->breakdowns++;
                    }
                } else if (method == ORC_CWY) {
                    /* Alg. 4 with the new implementation of Sec. 3.3.2 */
                    int broke;
                    for (int64_t i = jc + 1; i < mcmax; ++i) T[i + jc * mcmax] = 0.0;
                    double fl = 0.0;
                    double c = cwy_new_step(n, jc, Y, T, mcmax, v, q, work, &broke, &fl);
                    if (st) st->orth_flops += fl;
                    for (int64_t r = 0; r < n; ++r) v[r] = -c * q[r];
                    if (broke) {
                        success_allowed = 0;
                        if (st) st->breakdowns++;
                    }
                } else {
                    /* Householder orthogonalization (Alg. 2) applied to this iterate */
                    int64_t hf = 0;
                    for (int64_t i = 0; i < jc; ++i) hf += apply_reflector(n, i, Y + i * n, tv[i], v);
                    double* yk = Y + jc * n;
                    for (int64_t r = 0; r < jc; ++r) yk[r] = 0.0;
                    int broke;
                    double c = reflector(n - jc, v + jc, yk + jc, &broke);
                    tv[jc] = 2.0 / dot(n - jc, yk + jc, yk + jc);
                    for (int64_t r = 0; r < n; ++r) q[r] = 0.0;
                    q[jc] = 1.0;
                    for (int64_t i = jc; i >= 0; --i) hf += apply_reflector(n, i, Y + i * n, tv[i], q);
                    for (int64_t r = 0; r < n; ++r) v[r] = c * q[r];
                    if (st) st->orth_flops += 2.0 * (double)hf;
                    if (broke) {
                        success_allowed = 0;
                        if (st) st->breakdowns++;
                    }
                }
            }
            /* convergence test on ||x||_inf (DSTEIN) */
            double nrm = 0.0;
            for (int64_t r = 0; r < n; ++r) nrm = dmax(nrm, fabs(v[r]));
            if (success_allowed && nrm >= dtpcrt) {
                nrmchk++;
                if (nrmchk >= EXTRA + 1) {
                    converged = 1;
                    break;
                }
            }
        }
        if (st) st->sweeps += its;
        if (iters) iters[j] = its;
        if (!converged) {
            if (ifail) ifail[info] = j;
            info++;
        }
        /* Alg. 1 / Alg. 4: normalize; the first entry of largest magnitude
           is made positive (DSTEIN's convention). */
        double nr = nrm2(n, v);
        int64_t jmax = 0;
        for (int64_t r = 1; r < n; ++r)
            if (fabs(v[r]) > fabs(v[jmax])) jmax = r;
        double scl = 1.0 / nr;
        if (v[jmax] < 0.0) scl = -scl;
        double* zj = Z + j * ldz;
        for (int64_t r = 0; r < n; ++r) zj[r] = scl * v[r];
    }

    free(wp);
    free(head);
    free(u0);
    free(u1);
    free(u2);
    free(l);
    free(piv);
    free(v);
    free(q);
    free(work);
    free(Y);
    free(T);
    free(tv);
    return info;
}

/* ------------------------------------------------------------------------------------ */
/* Cyclic Jacobi (Golub & Van Loan, Matrix Computations, cyclic-by-row Jacobi)             */
/* ------------------------------------------------------------------------------------ */

void orc_jacobi(int64_t n, double* A, double* lam, double* V)
{
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) V[i + j * n] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) {
                double a = A[i + j * n] * A[i + j * n];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-34 * tot || off == 0.0) break;
        for (int64_t p = 0; p < n - 1; ++p)
            for (int64_t qq = p + 1; qq < n; ++qq) {
                double apq = A[p + qq * n];
                if (apq == 0.0) continue;
                double app = A[p + p * n], aqq = A[qq + qq * n];
                /* symmetric Schur 2x2: tau = (a_qq - a_pp)/(2 a_pq), t = sgn/(|tau|+sqrt(1+tau^2)) */
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- J^T A J with J = rotation in the (p,q) plane */
                for (int64_t k = 0; k < n; ++k) {
                    double akp = A[k + p * n], akq = A[k + qq * n];
                    A[k + p * n] = c * akp - s * akq;
                    A[k + qq * n] = s * akp + c * akq;
                }
                for (int64_t k = 0; k < n; ++k) {
                    double apk = A[p + k * n], aqk = A[qq + k * n];
                    A[p + k * n] = c * apk - s * aqk;
                    A[qq + k * n] = s * apk + c * aqk;
                }
                for (int64_t k = 0; k < n; ++k) {
                    double vkp = V[k + p * n], vkq = V[k + qq * n];
                    V[k + p * n] = c * vkp - s * vkq;
                    V[k + qq * n] = s * vkp + c * vkq;
                }
            }
    }
    /* sort ascending (selection sort, columns of V follow) */
    for (int64_t i = 0; i < n; ++i) lam[i] = A[i + i * n];
    for (int64_t i = 0; i < n; ++i) {
        int64_t kmin = i;
        for (int64_t k = i + 1; k < n; ++k)
            if (lam[k] < lam[kmin]) kmin = k;
        if (kmin != i) {
            double t = lam[i];
            lam[i] = lam[kmin];
            lam[kmin] = t;
            for (int64_t r = 0; r < n; ++r) {
                double tmp = V[r + i * n];
                V[r + i * n] = V[r + kmin * n];
                V[r + kmin * n] = tmp;
            }
        }
    }
}
