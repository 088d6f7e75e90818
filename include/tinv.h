/*
 * tinv.h -- C ABI of the GB300 (sm_103a) library for all eigenvectors of a real symmetric
 * tridiagonal matrix by inverse iteration with compact-WY (or MGS) reorthogonalization.
 *
 * Method: Ishigami, Kimura, Nakamura, "On Implementation and Evaluation of Inverse Iteration
 * Algorithm with compact WY Orthogonalization", arXiv:1209.1910.  Problem statement Sec. 2.1
 * (Eq. 1); classical inverse iteration Alg. 1; DSTEIN-cWY Alg. 4 with the compact-WY update
 * of Sec. 3.3.2 (Eqs. yt, cwy1, cwy2).
 *
 * Conventions shared by every entry point:
 *   - T is given by its diagonal d[0..n) and off-diagonal e[0..n-1) (e may be NULL if n == 1).
 *   - Eigenvalue approximations w[0..m) must be finite and ascending (non-decreasing).
 *   - Matrices are column-major with a leading dimension (ldz >= n, ldv >= n).
 *   - All arithmetic is IEEE binary64.
 *   - Unless tinv_opts.device_ptrs is set, every pointer is HOST memory owned by the caller;
 *     the call copies inputs to the GPU, runs, copies results back and synchronizes.
 *     With device_ptrs set, every array pointer is DEVICE memory of the current device, the
 *     work is enqueued on tinv_opts.stream and the call returns without synchronizing, except
 *     where an entry point says otherwise (tinv_split, tinv_eig, tinv_bdsvd and tinv_tune form
 *     host-side tables or timings; any call given tinv_opts.phase_ms).
 *   - Return codes: 0 = success; -k = argument k is invalid (1-based position in the call);
 *     > 0 = number of eigenvectors that did not converge within MAXITS = 5 sweeps (their
 *     columns are still written, as LAPACK DSTEIN does); values <= -100 are runtime errors
 *     listed below.  tinv_strerror() gives a message for any code.
 *   - Thread safety: calls on different streams may run concurrently from different host
 *     threads; the library keeps no global mutable state besides a per-device cache of the
 *     number of SMs, the tune cache of tinv_tune (guarded by a lock), and the shared scratch
 *     of tinv_solve_noalloc (see there).
 */
#ifndef TINV_H
#define TINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TINV_OK 0
#define TINV_ENOMEM (-101)    /* device or pinned-host allocation failed                   */
#define TINV_ECUDA (-102)     /* a CUDA runtime call failed (launch, copy, sync)           */
#define TINV_ETIMEDOUT (-103) /* a bounded device-side wait expired (see each kernel)      */
#define TINV_EAGAIN (-104)    /* server: no slot / memory free right now, retry            */
#define TINV_ECANCELED (-105) /* server: request was cancelled                            */
#define TINV_ENOTSUP (-106)   /* size beyond what this library supports                    */
#define TINV_ENODEV (-107)    /* no CUDA device, or not an sm_103 device                   */
#define TINV_EWORKSPACE (-108) /* caller-provided workspace is too small                   */
#define TINV_EINTERNAL (-109) /* a device-side bounds check failed (TINV_DEBUG builds only)  */

/* Reorthogonalization of eigenvectors inside a cluster. */
#define TINV_CWY 0 /* compact-WY Householder orthogonalization (Sec. 3.3.2, Alg. 4)   */
#define TINV_MGS 1 /* modified Gram-Schmidt as in LAPACK DSTEIN (Alg. 1)               */

typedef struct tinv_opts {
    int32_t method;      /* TINV_CWY (default) or TINV_MGS                                   */
    int32_t device_ptrs; /* 0: host pointers, synchronous; 1: device pointers, async         */
    void* stream;        /* cudaStream_t used when device_ptrs = 1 (NULL = legacy stream)    */
    uint64_t seed;       /* start vectors: counter-based SplitMix64 keyed by (seed, j0 + j)  */
    int64_t j0;          /* index offset of w[0] inside a larger problem (for start keys)    */
    void* workspace;     /* optional device workspace (device_ptrs = 1); NULL = the library  */
    size_t workspace_bytes; /*   allocates stream-ordered memory itself, from a memory pool   */
                            /*   of its own per device and context that keeps freed memory  */
                            /*   for later calls (no pool is created during graph capture)  */
    int32_t* iters;      /* optional [m]: sweeps taken by vector j, negated if not converged;  */
                         /*   host or device memory following device_ptrs                     */
    int64_t* info;       /* optional (device_ptrs = 1): device scalar that receives the count */
                         /*   of non-converged vectors                                         */
    int32_t max_team;    /* 0 = automatic; otherwise the most CTAs one cluster may use        */
    int32_t grid_ctas;   /* 0 = all co-resident CTAs; otherwise cap on the persistent grid    */
    float* phase_ms;     /* optional HOST [4]: device milliseconds of the plan, LU, first-sweep */
                         /*   and cluster kernels, from CUDA events on the call's stream; the  */
                         /*   call then synchronizes that stream before returning             */
    int64_t* counters;   /* optional [4], host or device memory following device_ptrs: [0]   */
                         /*   cluster-kernel solves whose back substitution was redone         */
                         /*   sequentially (consistency check failed), [1] clusters with >= 2  */
                         /*   members, [2] clusters given CTA teams, [3] as [0] for the first   */
                         /*   sweeps                                                            */
    int32_t table_ready; /* tinv_batch with device pointers and o->workspace: 1 = the workspace */
                         /*   already holds this batch's problem table (an earlier call with    */
                         /*   the same n, off_de, off_z, seed and j0 wrote it); the call then   */
                         /*   makes no host-to-device copy and no allocation, so it can be      */
                         /*   captured into a CUDA graph and replayed (phase_ms must be NULL)   */
    int32_t spin_limit;  /* polls after which a bounded team-barrier wait of the cluster kernel  */
                         /*   gives up (0 = the default: 4e8 polls or 20 s, whichever is first); */
                         /*   a small value makes a launch end with TINV_ETIMEDOUT, which tests  */
                         /*   the bounded-wait failure path without hanging the GPU              */
    int32_t block;       /* compact WY only: 0 or 1 = each cluster member orthogonalized on its  */
                         /*   own (Alg. 4); b = 2..16 = a cluster's members after its head in   */
                         /*   blocks of up to b that sweep together and are orthogonalized by   */
                         /*   the compact-WY block form of Sec. 3.2 (Eqs. cwy1/cwy2).  Applies  */
                         /*   to clusters of >= 3 members on CTA teams (the block is at most    */
                         /*   twice the team size); clusters on single CTAs take b = 1          */
    int32_t reserved[3];
} tinv_opts;

/* Fill *o with the defaults: CWY, host pointers, seed 0, j0 0, automatic scheduling. */
void tinv_opts_default(tinv_opts* o);

/* Human-readable message for a return code. */
const char* tinv_strerror(int code);

/* Library version string and the CUDA architecture it was built for. */
const char* tinv_version(void);

/*
 * tinv -- all n eigenvectors of T (Sec. 2.1: compute v_j for every lambda_j).
 *   n   : matrix order, n >= 0 (n = 0 is a no-op; n = 1 gives Z = [1]).
 *   d,e : host arrays [n], [n-1].
 *   w   : host array [n], ascending eigenvalue approximations (e.g. from bisection).
 *   Z   : host array n x n, column-major, ldz = n, caller-allocated; column j receives the
 *         unit eigenvector of w[j], sign chosen so its first entry of largest magnitude is
 *         positive.
 * Defaults of tinv_opts_default() apply (CWY, seed 0).  Returns as described above.
 */
int tinv(int64_t n, const double* d, const double* e, const double* w, double* Z);

/*
 * tinv_ex -- eigenvectors of m eigenvalues w[0..m) (m <= n), with options.
 *   Arguments as tinv; Z is n x m with leading dimension ldz >= n.
 *   ifail : optional host array [m]; on return its first r entries are the (0-based) indices
 *           of the r vectors that did not converge (host-pointer mode only).
 *   o     : options (NULL = defaults).  With o->device_ptrs the call is asynchronous on
 *           o->stream and returns 0 when the work is enqueued; the non-converged count goes
 *           to o->info and per-vector sweep counts to o->iters.
 * Clusters are found by the Peters-Wilkinson test |w'_j - w'_{j-1}| <= 1e-3 ||T||_1 over the
 * perturbed shifts w' (Sec. 2.1; Alg. 1 / Alg. 4).
 */
int tinv_ex(int64_t n, const double* d, const double* e, int64_t m, const double* w, double* Z,
            int64_t ldz, const tinv_opts* o, int64_t* ifail);

/* Bytes of device workspace tinv_ex needs for (n, m) with the given options. */
size_t tinv_workspace_size(int64_t n, int64_t m, const tinv_opts* o);

/*
 * tinv_tune -- autotuner for the cluster kernel's team cap (tinv_opts.max_team) on one problem.
 * A cluster's member sweeps (Alg. 4; the passes of Sec. 3.3.2 and the solve) are split over a
 * team of CTAs that meet at team barriers: a larger team has more FP64 units and waits longer for
 * its slowest CTA.  The automatic rule sizes teams by each cluster's share of the m_c^2 n work;
 * tinv_tune measures instead.  It runs tinv_ex on the problem once per candidate cap (the
 * automatic rule, then 2, 4, 8, ... below the grid, n/16 and 192), one warm-up call and `reps`
 * timed calls each (CUDA events on its own stream), and keeps the automatic rule unless a cap is
 * at least 1% faster.
 *   n, d, e, m, w : the problem, as for tinv_ex; host or device memory per o->device_ptrs (with
 *            host pointers the values are checked as tinv_ex checks them).
 *   o      : options (NULL = defaults).  method, seed, j0 and grid_ctas are those tuned for;
 *            max_team, workspace, iters, info, counters, phase_ms and stream are not used.
 *   reps   : timed calls per candidate, >= 1.
 *   max_team : out, the chosen cap (0 = the automatic rule); pass it as tinv_opts.max_team in
 *            later calls on problems of this shape.
 *   ms     : optional out, mean device milliseconds of one call with the chosen cap.
 *   cached : optional out, 1 when the choice came from the tune cache and nothing was run.
 * Tune cache: choices are kept for the life of the process (thread-safe), keyed by the device's
 * name and SM count, method, grid cap, n, m, the number of clusters with >= 2 members and the
 * largest cluster (from the plan of step a2, tinv_plan).  A call whose key is cached returns that
 * choice after the plan alone.  tinv_tune_clear() empties the cache; tinv_tune_save/_load write
 * and read it as a text file.  If the environment variable TINV_TUNE_CACHE names a file, the
 * first tinv_tune call of the process merges that file into the cache, and every new choice
 * rewrites the file (best effort: a file that cannot be written is not an error of the call).
 * The call is synchronous in both pointer modes; it allocates its own Z and workspace (the
 * device memory of one tinv_ex call with host pointers) and frees them before returning.
 * Returns 0; -1 n < 0; -2 d; -3 e; -4 m outside [0, n]; -5 w (NULL; with host pointers also
 * non-finite or not ascending); -6 method; -7 reps < 1; -8 max_team NULL; or a runtime code.
 */
int tinv_tune(int64_t n, const double* d, const double* e, int64_t m, const double* w,
              const tinv_opts* o, int32_t reps, int32_t* max_team, float* ms, int32_t* cached);

/* Result of tinv_tune_auto / tinv_tune_batch. */
typedef struct tinv_tuning {
    int32_t max_team; /* chosen team cap (tinv_opts.max_team; 0 = the automatic rule)            */
    int32_t block;    /* chosen block (tinv_opts.block; 0 = one member at a time)                */
    float ms;         /* mean device milliseconds of one call with the choice                    */
    int32_t cached;   /* 1 when the choice came from the tune cache and nothing was run           */
    int32_t reserved[4];
} tinv_tuning;

/*
 * tinv_tune_auto -- tinv_tune over both launch parameters of the cluster kernel: the switch
 * between one member at a time (Sec. 3.3.2, GEMV passes) and the blocked compact-WY form of
 * Sec. 3.2 (tinv_opts.block 4, 8 or 16, passes over Y for several members at once), then the team
 * cap with the chosen block.  Each stage keeps the current choice unless a candidate is at least
 * 1% faster; MGS and problems without multi-member clusters take (0, 0).  Arguments as
 * tinv_tune (o->block and o->max_team are not used); *out receives the choice.  Cached like
 * tinv_tune under a key of its own.  Returns as tinv_tune, with -8 for out == NULL.
 */
int tinv_tune_auto(int64_t n, const double* d, const double* e, int64_t m, const double* w,
                   const tinv_opts* o, int32_t reps, tinv_tuning* out);

/*
 * tinv_tune_batch -- the same two-stage search for a batch (tinv_batch), timing tinv_batch on the
 * caller's problems.  Arguments as tinv_batch (d, e, w host or device memory per o->device_ptrs;
 * n, off_de, off_z host arrays); reps timed calls per candidate.  The tune cache key is the
 * batch's size profile: device, SM count, method, grid cap, the total order, the number of
 * problems, a 62-bit hash of the count of problems in each power-of-two order class, and the
 * largest order.  The call allocates its own Z, info and workspace and synchronizes.  Returns 0;
 * -1 nprob < 0; -2 n; -3 off_de; -4 off_z (NULL or negative); -5 d; -6 e; -7 w (NULL; with
 * host pointers also non-finite or not ascending); -8 method; -9 reps < 1; -10 out NULL; or a
 * runtime code.
 */
int tinv_tune_batch(int64_t nprob, const int64_t* n, const int64_t* off_de, const int64_t* off_z,
                    const double* d, const double* e, const double* w, const tinv_opts* o,
                    int32_t reps, tinv_tuning* out);

/* Empty the tune cache of tinv_tune, tinv_tune_auto and tinv_tune_batch. */
void tinv_tune_clear(void);

/*
 * tinv_tune_save -- write the tune cache to `path` (created or truncated): a tag line
 * "# tinv tune cache v2", then one entry per line with tab-separated fields: kind (0 tinv_tune,
 * 1 tinv_tune_auto, 2 tinv_tune_batch), device name, SM count, method, grid cap, the options'
 * block, n, m, clusters with >= 2 members (batch: size-profile hash), largest cluster (batch:
 * largest order), chosen cap, chosen block, milliseconds.  Returns 0, -1 (path NULL) or -2 (the
 * file cannot be written).
 */
int tinv_tune_save(const char* path);

/*
 * tinv_tune_load -- merge the entries of a file written by tinv_tune_save into the tune cache
 * (an entry with the same key is replaced); files with the v1 tag (no kind and no block fields)
 * are read as tinv_tune entries with block 0.  Returns the number of entries read (>= 0), -1
 * (path NULL), -2 (the file cannot be read or lacks a tag line) or -3 (a malformed entry -- a
 * missing or non-numeric field, trailing text, a line longer than 1023 bytes, or a value out of
 * range: unknown kind, SM count <= 0, m > n or largest cluster > m (kinds 0 and 1), cap outside
 * [0, 192], block outside [0, 16], time negative or not finite, unknown method; the entries before
 * it are kept, the rest of the file is not read).  No device is needed.
 */
int tinv_tune_load(const char* path);

/*
 * tinv_batch -- all eigenvectors of nprob independent problems of uneven order, computed together
 * by one launch sequence: each problem is Sec. 2.1's problem (every lambda_j of its T), solved as
 * tinv_ex would solve it alone; clusters never span problems, and the clusters and eigenvalues of
 * all problems share the persistent kernels' work (large clusters get CTA teams, the rest are
 * queued largest first).
 *   nprob   : number of problems, >= 0 (0 is a no-op).
 *   n       : HOST array [nprob], order of each problem (>= 0).
 *   off_de  : HOST array [nprob], offset of problem q's entries in the packed d, e and w arrays:
 *             d[off_de[q] .. +n[q]), e[off_de[q] .. +n[q]-1), w[off_de[q] .. +n[q]) (ascending).
 *   off_z   : HOST array [nprob], offset of problem q's eigenvector matrix in the packed Z array:
 *             n[q] x n[q], column-major, leading dimension n[q].  Regions must not overlap.
 *   d, e, w : packed inputs;  Z : packed outputs (caller-allocated).
 *   info    : optional [nprob]: per problem, the number of vectors that did not converge, or
 *             TINV_ETIMEDOUT for every problem if a bounded device wait expired.
 *   o       : options as tinv_ex (method, seed and j0 apply to every problem, so each problem gets
 *             the start vectors, and hence the result, of a tinv_ex call with the same options);
 *             o->iters, if given, has sum(n) entries in problem order.
 * d, e, w, Z, info and o->iters are host or device memory following o->device_ptrs; n, off_de
 * and off_z are always host memory (the workspace layout depends on them).  With device pointers
 * the call is asynchronous on o->stream (the problem table is copied from host memory first).
 * Returns 0, -k for an invalid argument k (a problem with non-finite or non-ascending inputs is
 * reported as its array's argument), the total number of non-converged vectors (> 0), or a
 * runtime error code.
 */
int tinv_batch(int64_t nprob, const int64_t* n, const int64_t* off_de, const int64_t* off_z,
               const double* d, const double* e, const double* w, double* Z, int64_t* info,
               const tinv_opts* o);

/* Bytes of device workspace tinv_batch needs for the problem orders n[0..nprob). */
size_t tinv_batch_workspace_size(int64_t nprob, const int64_t* n, const tinv_opts* o);

/*
 * tinv_bisect -- all n eigenvalues of T, ascending, by Sturm-count bisection (the eigenvalue step
 * that precedes inverse iteration; the paper computes it with LAPACK's bisection, Sec. 5.1).
 *   d, e : T as above;  w : [n] receives the eigenvalue approximations, ascending.
 * Eigenvalue k is halved from the Gershgorin interval (widened by 2 eps n max|bound| + 2 pivmin)
 * until the bracket is at most max(2 eps max(|lo|,|hi|), eps ||T||_1), and the midpoint is
 * returned; a pivot of the Sturm sequence smaller than pivmin = DBL_MIN max(1, max e_i^2) in
 * magnitude counts as -pivmin.  Each eigenvalue is computed independently, with IEEE binary64
 * round-to-nearest operations in a fixed order, so results do not depend on the launch.
 * Pointers follow o->device_ptrs (NULL o: host pointers, synchronous).
 * Returns 0, -k for invalid argument k, or a runtime error code.
 */
int tinv_bisect(int64_t n, const double* d, const double* e, double* w, const tinv_opts* o);

/*
 * tinv_bisect_batch -- tinv_bisect for nprob problems in one launch.  n, off_de are HOST arrays
 * as for tinv_batch; problem q's eigenvalues go to w[off_de[q] .. +n[q]), so w is ready to be
 * passed to tinv_batch.  At most 65535 problems per call (else TINV_ENOTSUP).
 */
int tinv_bisect_batch(int64_t nprob, const int64_t* n, const int64_t* off_de, const double* d,
                      const double* e, double* w, const tinv_opts* o);

/*
 * tinv_split -- the unreduced blocks of T.  The paper takes its eigenvalues from LAPACK's
 * bisection (Sec. 5.1), which hands DSTEIN the blocks of T (IBLOCK/ISPLIT); the rule here: row i
 * ends a block iff |e_i| <= eps ||T||_1, with eps = 2^-52 and ||T||_1 = max_i(|d_i| + |e_{i-1}|
 * + |e_i|) (dropping such an entry changes T by at most eps ||T||_1 in norm).
 *   isplit : [n] receives, for each block b < *nblock, one past its last row (ascending; the last
 *            entry is n).  nblock : receives the number of blocks (0 for n = 0).
 * d, e and isplit follow o->device_ptrs for d, e only: isplit and nblock are always host memory
 * (the call synchronizes o->stream).  Returns 0, -k for invalid argument k, or a runtime error.
 */
int tinv_split(int64_t n, const double* d, const double* e, int64_t* isplit, int64_t* nblock,
               const tinv_opts* o);

/*
 * tinv_eig -- all eigenvalues and eigenvectors of T, with T split first (tinv_split): each block
 * is an independent problem whose eigenvalues come from bisection (tinv_bisect) and whose
 * eigenvectors come from inverse iteration with the chosen reorthogonalization (tinv_batch over
 * the blocks; method, seed and j0 apply to every block as in tinv_batch).  The block results are
 * merged into ascending order by a stable sort over the blocks' eigenvalues taken in block order
 * (equal values keep the lower block first).
 *   w      : [n] receives the eigenvalues, ascending.
 *   Z      : n x n, column-major, leading dimension ldz >= n: column j receives the unit
 *            eigenvector of w[j] (sign as in tinv), exactly zero outside its block.
 *   iblock : optional [n]: the block (0-based) of each eigenvalue.
 *   isplit, nblock : optional, as tinv_split (always host memory).
 *   o      : method, seed, j0, max_team, grid_ctas apply; o->iters, if given, receives the sweep
 *            counts in the order of w; o->phase_ms, if given, receives the device times of the
 *            inverse-iteration launches as for tinv_batch; workspace and counters are not used.
 * d, e, w, Z, iblock and o->iters are host or device memory following o->device_ptrs.  The call
 * synchronizes o->stream (the block table and the merge order are formed on the host).
 * Returns 0, -k for invalid argument k (n = 1, d = 2, e = 3, w = 4, Z = 5, ldz = 6, method = 10),
 * the total number of non-converged vectors (> 0), or a runtime error code.
 */
int tinv_eig(int64_t n, const double* d, const double* e, double* w, double* Z, int64_t ldz,
             int64_t* iblock, int64_t* isplit, int64_t* nblock, const tinv_opts* o);

/*
 * tinv_bdsvd -- singular triplets of an upper bidiagonal B (diagonal a[n], superdiagonal b[n-1])
 * by this inverse iteration applied to B's Golub-Kahan form (singular vectors of a bidiagonal
 * matrix are named as a further use of the method in Sec. 6): T_GK of order 2n has zero diagonal
 * and off-diagonal (a_1, b_1, a_2, b_2, ..., a_n); its eigenvalues are +-sigma_i and the
 * eigenvector of +sigma is (v_1, u_1, ..., v_n, u_n)/sqrt(2).  The n largest eigenvalues of T_GK
 * come from bisection (tinv_bisect), their eigenvectors from tinv_ex with the chosen method, and
 * each vector's even and odd entries, scaled to unit length separately (a half that is all zero
 * stays zero), give v_j and u_j.
 *   s     : [n] receives the singular values, ascending.
 *   U, V  : n x n, column-major, leading dimensions ldu, ldv >= n: B v_j = s_j u_j and
 *           B^T u_j = s_j v_j.  Rows n .. ld-1 of each column are not written.
 *   o     : method, seed, j0 (keys of the start vectors of T_GK's eigenvectors, as tinv_ex),
 *           max_team and grid_ctas apply; o->iters, if given, receives the n sweep counts;
 *           o->phase_ms, if given, receives the device times of the inverse-iteration launches
 *           as for tinv_ex; workspace and counters are not used.
 * A zero singular value (a singular B) has a two-dimensional eigenspace in T_GK whose vectors
 * need not split into a v and a u of equal weight; its columns are then not reliable.
 * a, b, s, U, V and o->iters follow o->device_ptrs; the call synchronizes o->stream.
 * Returns 0, -k for invalid argument k (n = 1, a = 2, b = 3, s = 4, U = 5, ldu = 6, V = 7,
 * ldv = 8, method = 9), the number of non-converged vectors (> 0), or a runtime error code.
 */
int tinv_bdsvd(int64_t n, const double* a, const double* b, double* s, double* U, int64_t ldu,
               double* V, int64_t ldv, const tinv_opts* o);

/*
 * tinv_plan -- step a1/a2 alone (Sec. 2.1; Alg. 4): ||T||_1, the cluster
 * tolerance, the convergence threshold and the cluster head of every eigenvalue.
 *   wp    : [m] perturbed shifts w' (coincident approximations are separated by 10 eps |w|).
 *   head  : [m] index of the first member of the cluster of j (j itself for a cluster head).
 *   scal  : [3] = { ||T||_1, 1e-3 ||T||_1, sqrt(0.1/n) }.
 * Pointers follow o->device_ptrs.  Deterministic and bit-identical to a sequential scan.
 */
int tinv_plan(int64_t n, const double* d, const double* e, int64_t m, const double* w,
              double* wp, int32_t* head, double* scal, const tinv_opts* o);

/*
 * tinv_lu -- step a3 alone: LU with scaled partial pivoting of T - s_j I (the matrix of Eq. 1;
 * rows k+1 and k are interchanged when |c_k|/(|c_k|+|a_{k+1}|+|b_{k+1}|) > |a_k|/(|a_k|+|b_k|)
 * with the current pivot row's entries a_k, b_k; ties keep the row) for every shift s[0..m).
 * Outputs are m x n arrays, row j (stride n) for shift j:
 *   l     : multipliers of the unit lower bidiagonal L;  u0 : diagonal of U;
 *   u1,u2 : first and second superdiagonals of U;  piv : 1 where rows k, k+1 were swapped.
 * Entries past the end of each factor (l, u1, u2 at k = n-1, u2 at n-2) are written as 0.
 * Bit-identical to a sequential evaluation with the same operation order (no contraction).
 */
int tinv_lu(int64_t n, const double* d, const double* e, int64_t m, const double* s, double* l,
            double* u0, double* u1, double* u2, uint8_t* piv, const tinv_opts* o);

/*
 * tinv_solve -- step a5 alone: x_j <- (T - s_j I)^{-1} x_j for m right-hand sides X (n x m,
 * ldx), each scaled first as in DSTEIN when scale != 0 (x <- x n ||T||_1 max(eps,|u_nn|)/||x||_1).
 * A diagonal entry u of U so small that a quotient of its row by it could overflow
 * (|u| < DBL_MIN max(1, |u1|, |u2|), zero included) is replaced by sign(u) tol, tol = eps max|U|
 * (DLAGTS's perturbation, made only to avoid overflow).
 */
int tinv_solve(int64_t n, const double* d, const double* e, int64_t m, const double* s,
               double* X, int64_t ldx, int32_t scale, const tinv_opts* o);

/*
 * tinv_solve_noalloc -- tinv_solve for device pointers that allocates no memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot have a library allocate device
 * memory, e.g. code whose device memory is all owned by a framework's caching allocator or by a
 * fixed arena, or code on a path where the implicit synchronization of cudaMalloc/cudaFree is
 * not acceptable.
 *   n, d, e, m, s, X, ldx, scale : as tinv_solve; d, e, s and X are DEVICE pointers of the
 *                                  current device.
 *   stream : cudaStream_t the work is enqueued on; the call returns without synchronizing.
 * Scratch: a fixed 20 MiB array in device memory, part of the library image (every GPU that
 * loads the library holds it until the process exits); it takes m * n <= 262144 and
 * m <= 131072 (for example 512 shifts of order 512).  Larger sizes return TINV_ENOTSUP.  The
 * call performs no cudaMalloc or cudaFree.  The first call in a CUDA context (the device's
 * primary context, or a driver context the caller made current) looks up the array's device
 * address in that context and caches it under the context's unique id; make that first call
 * before any stream capture.  All calls on a device share the array and it keeps the last call's
 * contents (each call writes every entry it reads), so calls whose work overlaps on the GPU race:
 * serialize them, e.g. on one stream.  X is written only in its rows [0, n) of each of its m
 * columns; the rows n..ldx-1 are left untouched.
 */
int tinv_solve_noalloc(int64_t n, const double* d, const double* e, int64_t m, const double* s,
                       double* X, int64_t ldx, int32_t scale, void* stream);

/*
 * tinv_orth -- incremental orthogonalization of the columns of V (n x m, ldv) by the GPU
 * reorthogonalization kernels, without inverse iteration (Sec. 3):
 *   method TINV_CWY: Alg. 3 in the form of Sec. 3.3.2; Q[:,j] = (Y_j T_j Y_j^T - I) e_j (the
 *                    sign-flipped q_j of that section); optional Y (n x m, ld n) and T
 *                    (m x m, ld m, upper triangular) receive the compact-WY factors.
 *   method TINV_MGS: modified Gram-Schmidt; Q[:,j] unit vectors; Y and T are not written.
 */
int tinv_orth(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q, int64_t ldq,
              double* Y, double* T, const tinv_opts* o);

/* ============================================================================================
 * Serving: a request queue with continuous batching.  The paper has no counterpart; it serves
 * many independent problems (each the problem of Sec. 2.1) arriving over time through the
 * batched path.  A worker thread owns the GPU: whenever one of its max_inflight streams is free
 * and at least one stream's share of the SMs (wave_ctas) is free, it forms a wave from the
 * pending requests and runs it (bisection for requests without eigenvalues, then the batched
 * inverse iteration of tinv_batch).  Requests are taken in arrival order until the wave holds
 * its share of the pending work (the free streams divide it; a request's work counts as n^3);
 * a request that does not fit max_slots or the memory budget right now is passed over, so
 * smaller requests behind it go first, but once 8 waves have passed it over it blocks the
 * requests behind it until it fits.  The memory budget is re-read at every admission:
 * hbm_fraction x (device memory free now + the estimate held by the server's waves in flight),
 * 57 n^2 + O(n) bytes per request.  The wave's persistent cluster kernel gets the free SMs in
 * proportion to its share of the pending work; a wave that empties the queue leaves one share
 * free for later arrivals while other streams are idle.  The grids of the waves in flight never
 * exceed the SM count, so their kernels are co-resident and overlap on the device, and a request
 * that arrives while others are on the GPU starts as soon as a stream, SMs and memory free up.
 * A problem's result does not depend on the other problems of its wave except through the CTA
 * team a large cluster gets (rounding only); with max_team = 1 it is bit-identical to a tinv_ex
 * call with the same seed.
 * ============================================================================================ */
typedef struct tinv_server tinv_server; /* opaque */

typedef struct tinv_server_cfg {
    int32_t max_slots;    /* most problems on the GPU at once (default 4096)                  */
    int32_t max_inflight; /* most waves in flight at once, one stream each (default 4, <= 8)  */
    double hbm_fraction;  /* share of the free device memory (re-read at each admission, plus  */
                          /*   what the server's waves hold) that waves may use (default 0.5,  */
                          /*   < 0.95); tinv_submit refuses a request above this share of the  */
                          /*   memory free at creation                                         */
    int32_t method;       /* TINV_CWY (default) or TINV_MGS                                    */
    int32_t max_team;     /* as tinv_opts.max_team                                             */
    int32_t max_pending;  /* queued requests beyond which tinv_submit returns TINV_EAGAIN      */
                          /*   (default 65536)                                                 */
    int32_t device;       /* CUDA device ordinal                                               */
    int32_t wave_ctas;    /* one stream's share of the SMs (persistent CTAs of a wave's       */
                          /*   cluster kernel, at least); 0 = the SM count / max_inflight      */
    int32_t block;        /* as tinv_opts.block (compact WY in blocks of members; 0 = off)     */
    int32_t reserved[6];
} tinv_server_cfg;

/* Request states (tinv_poll). */
#define TINV_REQ_PENDING 0   /* queued, not yet on the GPU              */
#define TINV_REQ_RUNNING 1   /* part of a wave on the GPU               */
#define TINV_REQ_DONE 2      /* Z written; tinv_wait returns its info   */
#define TINV_REQ_CANCELLED 3 /* cancelled; Z not written                */
#define TINV_REQ_FAILED 4    /* a runtime error; tinv_wait returns it   */

typedef struct tinv_stats {
    uint64_t submitted, completed, cancelled, failed, rejected;
    uint64_t waves;             /* waves launched                                         */
    uint64_t max_inflight_seen; /* most waves that were in flight at the same time         */
    uint64_t pending;           /* requests queued now                                    */
    uint64_t inflight_waves;    /* waves in flight now                                    */
    double mean_wave_problems;  /* problems per wave                                      */
    double p50_ms, p99_ms, mean_ms; /* submit-to-completion latency of completed requests */
    double problems_per_s;      /* completed requests / (last completion - first submit)  */
    double eigvecs_per_s;       /* completed eigenvectors over the same span               */
    double reserved[8];
} tinv_stats;

/* Fill *c with the defaults above. */
void tinv_server_cfg_default(tinv_server_cfg* c);

/* Start a server on cfg->device (NULL cfg = defaults): its streams and worker thread.  Returns
 * 0, -1 for an invalid configuration, -2 for a NULL out, or TINV_ENODEV / TINV_ECUDA. */
int tinv_server_create(const tinv_server_cfg* cfg, tinv_server** out);

/* Queue the problem (n, d, e) for all n eigenvectors.  d, e and w are HOST arrays copied before
 * the call returns; w (ascending) may be NULL, and the eigenvalues are then computed on the GPU
 * by tinv_bisect's bisection.  Z is a caller-owned HOST n x n buffer (column-major, ld n) that
 * must stay valid until the request is final; it is written only when the request completes.
 * seed keys the start vectors as tinv_opts.seed (with j0 = 0).  *ticket receives the request's
 * id.  Returns 0; -k for an invalid argument k (1-based); TINV_EAGAIN when max_pending requests
 * are queued (retry later); TINV_ENOTSUP when the problem alone exceeds the memory budget;
 * TINV_ECANCELED once the server is being destroyed. */
int tinv_submit(tinv_server* srv, int64_t n, const double* d, const double* e, const double* w,
                double* Z, uint64_t seed, uint64_t* ticket);

/* Current state (TINV_REQ_*) of a request; -2 if the ticket is unknown (never issued, or
 * already returned by tinv_wait). */
int tinv_poll(tinv_server* srv, uint64_t ticket, int32_t* state);

/* Wait until the request is final (timeout_ms < 0: without limit).  Returns 0 with *info = the
 * number of vectors that did not converge (LAPACK convention), TINV_ECANCELED, the runtime error
 * of a failed request, or TINV_ETIMEDOUT if the limit passed first (the request stays queued).
 * A final state releases the ticket. */
int tinv_wait(tinv_server* srv, uint64_t ticket, int32_t timeout_ms, int64_t* info);

/* Cancel a request: a pending one is removed from the queue at once; a running one finishes on
 * the GPU but its result is not written.  Returns 0 (Z will not be written by the server),
 * TINV_ECANCELED if it was already cancelled, 1 if it had already completed or its result is
 * being copied into Z (the request then completes normally and Z must stay valid until
 * tinv_wait returns), -2 for an unknown ticket. */
int tinv_cancel(tinv_server* srv, uint64_t ticket);

/* Counters and latency percentiles so far. */
int tinv_server_stats(tinv_server* srv, tinv_stats* st);

/* Finish every queued and running request (drain), then stop the worker and free the server.
 * No other call on srv may be in progress or follow. */
int tinv_server_destroy(tinv_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* TINV_H */
