// tinv_internal.h -- declarations shared by the kernel and host translation units of libtinv.
// Not part of the public ABI (that is include/tinv.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/tinv.h"

namespace tinvx {

constexpr int kFirstWarps = 8;      // warps per CTA of the warp-per-eigenvalue solve kernel
constexpr int kPlanThreads = 1024;  // threads of the single-CTA plan kernel
constexpr int kScalTeam = 16;       // doubles of per-CTA scalar partials
// Largest CTA team of the cluster kernel.  The distributed solve keeps, in the CTA's 2048-double
// scratch, 128 doubles of warp maps, 6 per rank of the maps published by the team and 6 x 128 of
// chunk maps: (2048 - 128 - 768) / 6 = 192 ranks.
constexpr int kTeamMax = 192;
// Largest block of the blocked compact-WY path (tinv_opts.block).
constexpr int kBlockMax = 16;

// Device error word bits.
constexpr int kErrTimeout = 1;   // a bounded spin wait expired
constexpr int kErrBounds = 2;    // a debug bounds check failed (TINV_DEBUG builds)

enum ChainMode : int32_t { kModeInvit = 0, kModeOrth = 1 };

// One independent tridiagonal problem of a launch (a whole tinv_ex call, or one problem of a
// batch).  Eigenvalues of all problems are numbered globally, problem by problem: problem s owns
// global indices [j0, j0 + m).  Its eigenvalue j has LU-factor rows (and, for cluster members,
// a Y column) of n entries at element offset foff + (j - j0) n of the factor arrays.
struct Seg {
    int64_t n;        // order
    int64_t m;        // number of eigenvalues / vectors
    int64_t de;       // offset of d[0] and e[0] in the packed d and e arrays
    int64_t wo;       // offset of w[0] in the packed w array
    int64_t z;        // offset of Z[0, 0] in the packed Z array
    int64_t ldz;      // leading dimension of this problem's Z
    int64_t j0;       // first global eigenvalue index
    int64_t foff;     // element offset of the factor rows / Y columns of eigenvalue j0
    int64_t kj0;      // start-vector key index of eigenvalue j0
    uint64_t seed;    // start-vector key seed
    double onenrm, ortol, dtpcrt;  // ||T||_1, 1e-3 ||T||_1, sqrt(0.1/n)   (written by the plan)
    double pad;
};

// Sizes a workspace is laid out for.
struct Dims {
    int64_t nmax;   // largest order of any problem
    int64_t M;      // total eigenvalues
    int64_t F;      // total factor elements: sum over problems of n m
    int64_t TT;     // elements reserved for T: sum over problems of m^2
    int64_t nseg;   // problems
    int32_t P;      // persistent grid size
    int32_t block;  // block size of the blocked compact-WY path (<= 1: none)
};
Dims single_dims(int64_t n, int64_t m, int32_t P, int32_t block = 0);
// tinv_opts.block as the layout uses it: 0 for MGS or b <= 1, else min(b, kBlockMax).
int32_t opts_block(const tinv_opts& o);

// Byte offsets of every device array inside one workspace allocation.
struct Layout {
    size_t segs, segj, sinfo;
    size_t scal, wp, head, clstart, clsize, cltoff, sched, queue, ctr, bar;
    size_t fl, fu1, fu2, fr, fpiv, u0n, tolv, rhs;
    size_t Y, T, partS, partG, partScal, vecS, vecX, vecR, qbuf, vbuf, tpub, gvec;
    size_t vblk, qblk, pblk, tblk;
    size_t total;
};

// Indices into the int64 counter block (ctr).
enum CtrIdx : int {
    kCtrNClust = 0,  // clusters with >= 2 members
    kCtrNQueue = 1,  // clusters processed by single CTAs from the queue
    kCtrQHead = 2,   // queue head (atomic)
    kCtrErr = 3,     // error word
    kCtrInfo = 4,    // non-converged vectors
    kCtrTSize = 5,   // entries of T used
    kCtrFallback = 6,       // cluster-kernel solves whose back substitution was redone sequentially
    kCtrFallbackFirst = 7,  // the same in the first-sweep kernel
    kCtrCount = 8
};

// Kernel arguments of a launch.  With seg_preset == 0 the problem table has one entry that
// the plan kernel fills from n, m, ldz, seed and j0; otherwise the table was copied into the
// workspace by the host before the launch.
struct Problem {
    int64_t n, m, ldz;  // single problem (seg_preset == 0); n = largest order otherwise
    const double* d;    // packed diagonals
    const double* e;    // packed off-diagonals
    const double* w;    // packed eigenvalue approximations
    double* Z;          // packed eigenvectors
    int32_t* iters;     // [M] or null
    int32_t method;
    int32_t seg_preset;
    uint64_t seed;
    int64_t j0;
    int64_t nseg, M;
    int64_t zlen;         // elements of the packed Z array the launch may touch (0 = unknown;
                          // used by the device bounds checks of TINV_DEBUG builds)
    uint32_t spin_limit;  // polls of a bounded team-barrier wait before it gives up (0 = the
                          // default kSpinLimit; tinv_opts.spin_limit, for testing the timeout path)
    uint32_t pad32;
};

// All device pointers derived from one workspace (see Layout).
struct Ws {
    Seg* segs;        // [nseg]
    int32_t* segj;    // [M]  problem of each global eigenvalue
    int64_t* sinfo;   // [nseg] non-converged vectors per problem
    double* scal;     // [4]  onenrm, ortol, dtpcrt of a single problem (tinv_plan)
    double* wp;       // [M]
    int32_t* head;    // [M]
    int32_t* clstart; // [M]
    int32_t* clsize;  // [M]
    int64_t* cltoff;  // [M]
    int32_t* sched;   // [P*4] team_first, team_size, team_rank, team_cluster
    int32_t* queue;   // [M]
    int64_t* ctr;     // [kCtrCount]
    uint32_t* bar;    // [P]
    double *fl, *fu1, *fu2, *fr;  // [F] LU factors, a row of n per eigenvalue
    uint8_t* fpiv;    // [F]
    double* u0n;      // [M]   |u_nn| before perturbation
    double* tolv;     // [M]   tiny-pivot threshold eps max|U| per shift
    double* rhs;      // [F]   right-hand sides kept for the sequential fallback (stand-alone
                      //       solve; the cluster path keeps them in Y)
    double* Y;        // [F]
    double* T;        // [TT]
    double *partS, *partG;  // [P*nmax]
    double* partScal;       // [P*kScalTeam]
    double *vecS, *vecX, *vecR, *qbuf;  // [P*nmax]
    double* vbuf;     // [P*nmax]  solved iterate of each team (rows of all CTAs)
    double* tpub;     // [P*8]  published solve maps of each team (2 + 6 doubles per rank)
    double* gvec;     // [P*2*nmax] global fallback for the per-CTA vectors (large n)
    int32_t P;        // persistent grid size the schedule was made for
    int32_t use_smem; // per-CTA vectors live in shared memory
    // extents in elements, for the device bounds checks of TINV_DEBUG builds
    int64_t nF;       // factor rows / Y columns (fl, fu1, fu2, fr, fpiv, Y, rhs)
    int64_t nTT;      // T
    int64_t nM;       // per-eigenvalue arrays
    int64_t nPN;      // per-CTA vectors and partials: P x nmax
    // blocked compact WY (block >= 2): per team slot (leader) kBlockMax vectors of nmax
    double* vblk;     // [P*kBlockMax*nmax] the block's iterates (solve outputs)
    double* qblk;     // [P*kBlockMax*nmax] the block's q vectors (next right-hand sides)
    double* pblk;     // [P*3*kBlockMax*nmax] per-CTA partial sums
    double* tblk;     // [P*3*kBlockMax*nmax] team vectors (G slots of a team)
    int32_t block;    // largest block (0: blocked path off)
    int32_t xcap;     // doubles of the block path's shared staging area
};

// Device bounds checks (TINV_DEBUG builds): a failed check sets kErrBounds in the error word
// and the caller skips the access and unwinds (no trap, no assert); team barriers see the error
// word and give up, so a whole launch ends and the host reports TINV_EINTERNAL.
#ifdef TINV_DEBUG
#define TINV_IN(cond, err) ::tinvx::dbg_ok((cond), (err))
#else
#define TINV_IN(cond, err) true
#endif

// need_chain: the cluster kernel's arrays; need_rhs: a copy of the right-hand sides (tinv_solve).
Layout make_layout(const Dims& D, bool need_chain, bool need_rhs = false);
Ws bind_layout(void* base, const Layout& L, const Dims& D);

// Kernel launchers (tinv_kernels.cu).  All enqueue on `st` and return cudaGetLastError().
cudaError_t launch_plan(const Problem& p, const Ws& w, int32_t max_team, cudaStream_t st);
// Norm and tolerances of a single problem only (into w.scal), for the stand-alone solve.
cudaError_t launch_norm(const Problem& p, const Ws& w, cudaStream_t st);
// LU of every eigenvalue's shifted matrix (problem table, perturbed shifts wp), solve-ready.
cudaError_t launch_lu_seg(const Problem& p, const Ws& w, cudaStream_t st);
// LU of T - shift_j I for all j.  With tolv != null the factors are made solve-ready in place
// (u0 -> r = 1/u0 with tiny pivots perturbed, u1 -> -u1 r, u2 -> -u2 r) and tolv[j] receives
// the tiny-pivot threshold; with tolv == null the factors are left as computed.
cudaError_t launch_lu(int64_t n, const double* d, const double* e, int64_t m, const double* shift,
                      double* l, double* u0_or_r, double* u1, double* u2, uint8_t* piv,
                      double* u0n, double* tolv, cudaStream_t st);
cudaError_t launch_first(const Problem& p, const Ws& w, cudaStream_t st);
cudaError_t launch_chain(const Problem& p, const Ws& w, int32_t mode, const double* V, int64_t ldv,
                         cudaStream_t st);
// Normalization and sign convention of the compact-WY cluster members (after launch_chain).
cudaError_t launch_finalize(const Problem& p, const Ws& w, cudaStream_t st);
cudaError_t launch_solve_rhs(int64_t n, int64_t m, const Ws& w, double* X, int64_t ldx,
                             int32_t scale, cudaStream_t st);
cudaError_t launch_orth_plan(const Problem& p, const Ws& w, int32_t method, cudaStream_t st);
cudaError_t launch_finish_info(const Problem& p, const Ws& w, int64_t* info_out, cudaStream_t st);

// Persistent-grid size (co-resident CTAs of the chain kernel) on the current device, and the
// threads per CTA it runs with.
int32_t chain_grid(int32_t cap, int64_t n);
int32_t chain_threads(int64_t n);
size_t chain_smem_bytes(int64_t n, bool use_smem, int32_t xcap = 0);
bool chain_use_smem(int64_t n);
// Shared staging capacity (doubles) of the blocked path for order n (0: blocking off).
int32_t block_xcap(int64_t n);

// Batched path on device arrays (tinv_api.cu): the device-pointer form of tinv_batch, with an
// optional per-problem seed array (host; null = o.seed for every problem).  Enqueues on
// o.stream; allocates its workspace stream-ordered unless o.workspace is given.
int batch_enqueue_device(int64_t nprob, const int64_t* n, const int64_t* off_de,
                         const int64_t* off_z, const uint64_t* seeds, const double* d,
                         const double* e, const double* w, double* Z, int64_t* info,
                         const tinv_opts& o);
size_t batch_workspace_bytes(int64_t nprob, const int64_t* n, const tinv_opts& o);

// Library status code of a device error word (kErrBounds before kErrTimeout).
inline int64_t err_code(int64_t err)
{
    if (err & kErrBounds) return TINV_EINTERNAL;
    return err ? (int64_t)TINV_ETIMEDOUT : 0;
}

// Library status code (include/tinv.h) of a CUDA runtime error.
inline int cuda_code(cudaError_t e)
{
    if (e == cudaSuccess) return TINV_OK;
    if (e == cudaErrorMemoryAllocation) return TINV_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
        e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDevice)
        return TINV_ENODEV;
    return TINV_ECUDA;
}

// True when the k host values are all finite (argument checks of host-pointer calls).
inline bool all_finite(const double* a, int64_t k)
{
    for (int64_t i = 0; i < k; ++i)
        if (!isfinite(a[i])) return false;
    return true;
}

// a[0..k) non-decreasing (NaN fails)
inline bool ascending(const double* a, int64_t k)
{
    for (int64_t i = 1; i < k; ++i)
        if (!(a[i] >= a[i - 1])) return false;
    return true;
}

// The library's stream-ordered memory pool on the current device and context (created on first
// use outside graph capture; it keeps freed memory instead of returning it at each
// synchronization, so the workspaces of repeated calls are not mapped again); null when there
// is none (no current context, or `st` is being captured before the pool exists).
cudaMemPool_t lib_pool(cudaStream_t st);
// Bytes the library's pool on the current device holds unused (free for its next allocations,
// though cudaMemGetInfo counts them as taken).
size_t lib_pool_idle();

// A device allocation owned by a scope: stream-ordered on `st` (from the library's pool, else
// the device's default pool, and cudaFreeAsync) when `use_async`, else cudaMalloc/cudaFree.
// Zero bytes allocate a small block.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    bool async = false;
    cudaError_t alloc(size_t bytes, cudaStream_t s, bool use_async)
    {
        st = s;
        async = use_async;
        if (bytes == 0) bytes = 256;
        if (!async) return cudaMalloc(&p, bytes);
        cudaMemPool_t pool = lib_pool(st);
        return pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMallocAsync(&p, bytes, st);
    }
    ~DevBuf()
    {
        if (!p) return;
        if (async)
            cudaFreeAsync(p, st);
        else
            cudaFree(p);
    }
};

// Sturm bisection of nprob problems (tinv_bisect.cu); ns/offs are DEVICE arrays, or null for
// one problem of order n1 at offset 0.  k0 > 0 (single problem only) computes eigenvalues
// k0 .. n1-1 alone, into w[k0 ..]; each index is bisected independently, so they are the same
// values a full call gives.
cudaError_t launch_bisect(int64_t nprob, const int64_t* ns, const int64_t* offs, int64_t n1,
                          int64_t nmax, const double* d, const double* e, double* w, cudaStream_t st,
                          int64_t k0 = 0);

}  // namespace tinvx
