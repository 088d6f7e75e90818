/*
 * tinv_oracle.h -- plain, slow, single-threaded CPU FP64 oracle for inverse iteration
 * with MGS / Householder / compact-WY reorthogonalization
 * (Ishigami, Kimura, Nakamura, "On Implementation and Evaluation of Inverse Iteration
 * Algorithm with compact WY Orthogonalization", arXiv:1209.1910).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this library. It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions: all matrices are column-major with an explicit leading dimension; all indices
 * are 0-based; "row r" of an n-vector is element r.  eps = DBL_EPSILON = 2^-52.
 */
#ifndef TINV_ORACLE_H
#define TINV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MGS = 0, ORC_CWY = 1, ORC_HOUSE = 2 };

/* Per-call statistics of orc_tinv (all optional). */
typedef struct {
    int64_t sweeps;        /* total inverse-iteration sweeps taken over all vectors      */
    int64_t breakdowns;    /* orthogonalizations whose remainder was exactly zero        */
    double  orth_flops;    /* flops spent in reorthogonalization (Table 1 accounting)    */
} orc_stats;

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the z-th output of the generator whose
 * state starts at `state` is orc_sm64_mix(state + z*gamma), z = 1, 2, ...               */
uint64_t orc_sm64_mix(uint64_t z);
uint64_t orc_sm64_next(uint64_t* state);
/* Counter-based start value in [-1, 1) for vector j, restart `attempt`, element i.      */
double orc_start_value(uint64_t seed, int64_t j, int attempt, int64_t i);

/* ||T||_1 = max_i (|d_i| + |e_{i-1}| + |e_i|) (the norm in the Peters-Wilkinson test). */
double orc_onenorm(int64_t n, const double* d, const double* e);

/* Split points: row i ends a block iff |e_i| <= eps ||T||_1; isplit[b] = one past the last row
 * of block b (isplit holds n entries).  Returns the number of blocks (0 for n = 0).     */
int64_t orc_split(int64_t n, const double* d, const double* e, int64_t* isplit);
/* Sturm count: number of eigenvalues of T strictly below x.                            */
int64_t orc_sturm_count(int64_t n, const double* d, const double* e, double x, double pivmin);
/* All n eigenvalues of T by Sturm-count bisection, ascending (the paper's DSTEBZ step). */
void orc_bisect(int64_t n, const double* d, const double* e, double* w);

/* Cluster plan over m ascending eigenvalue approximations w: perturbed shifts wp and
 * the index of each eigenvalue's cluster head (Peters-Wilkinson criterion).            */
void orc_plan(int64_t n, const double* d, const double* e, int64_t m, const double* w,
              double* wp, int64_t* head, double* onenrm, double* ortol, double* dtpcrt);

/* LU with scaled partial pivoting of T - lambda*I (Eq. 1's matrix).                    */
void orc_lagtf(int64_t n, const double* d, const double* e, double lambda,
               double* u0, double* u1, double* u2, double* l, unsigned char* piv);
/* Solve (T - lambda*I) x = y with the factors above; y is overwritten by x.            */
double orc_lagts(int64_t n, const double* u0, const double* u1, const double* u2,
                 const double* l, const unsigned char* piv, double* y);

/* Stand-alone incremental orthogonalizers: Q (n x m, ldq) from V (n x m, ldv).
 * Y (n x m) and T (m x m) receive the compact-WY factors where applicable (may be NULL). */
double orc_orth_mgs(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q, int64_t ldq);
double orc_orth_house(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q, int64_t ldq,
                      double* Y, double* tv);
double orc_orth_cwy_ordinary(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q,
                             int64_t ldq, double* Y, double* T);
double orc_orth_cwy_new(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q,
                        int64_t ldq, double* Y, double* T);

/* Alg. 3 with the columns taken nb at a time (Sec. 3.2): each block is orthogonalized against
 * the reflectors before it (Q^T = I - Y T^T Y^T), then by Householder QR of its own panel, and
 * T grows by Eq. cwy1.  Q, Y, T as orc_orth_cwy_new (Q holds the sign-flipped q_j).  Returns
 * the flops executed. */
double orc_orth_cwy_block(int64_t n, int64_t m, const double* V, int64_t ldv, int64_t nb,
                          double* Q, int64_t ldq, double* Y, double* T);

/* Inverse iteration for the m eigenvectors of w (DSTEIN structure, Alg. 1 for MGS,
 * Alg. 4 for CWY, Alg. 2 applied incrementally for HOUSE).  j0 offsets the index used
 * to key the random start vectors, so that a sub-range of a larger problem reproduces
 * the start vectors of the full problem.  Returns 0, or the number of vectors that did
 * not converge (their local indices in ifail, if given); iters[j] = sweeps of vector j. */
int64_t orc_tinv(int64_t n, const double* d, const double* e, int64_t m, const double* w,
                 int64_t j0, double* Z, int64_t ldz, int method, uint64_t seed,
                 int64_t* ifail, int32_t* iters, orc_stats* st);

/* orc_tinv's CWY iteration with each cluster's members after the head orthogonalized in blocks
 * of at most nb members spread evenly over the cluster (a block sweeps together; see
 * tinv_oracle.c).  nb = 1 is orc_tinv's CWY iteration. */
int64_t orc_tinv_blocked(int64_t n, const double* d, const double* e, int64_t m, const double* w,
                         int64_t j0, double* Z, int64_t ldz, int64_t nb, uint64_t seed,
                         int64_t* ifail, int32_t* iters, orc_stats* st);

/* Cyclic Jacobi on a dense symmetric n x n matrix A (overwritten): eigenvalues ascending
 * in lam, orthonormal eigenvectors in V (brute force for small n).                      */
void orc_jacobi(int64_t n, double* A, double* lam, double* V);

#ifdef __cplusplus
}
#endif
#endif
