// tinv_internal.h -- declarations shared by the kernel and host translation units of libtinv.
// Not part of the public ABI (that is include/tinv.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tinvx {

constexpr int kFirstWarps = 8;      // warps per CTA of the warp-per-eigenvalue solve kernel
constexpr int kPlanThreads = 1024;  // threads of the single-CTA plan kernel
constexpr int kScalTeam = 16;       // doubles of per-CTA scalar partials

// Device error word bits.
constexpr int kErrTimeout = 1;   // a bounded spin wait expired
constexpr int kErrBounds = 2;    // a debug bounds check failed (TINV_DEBUG builds)

enum ChainMode : int32_t { kModeInvit = 0, kModeOrth = 1 };

// Byte offsets of every device array inside one workspace allocation.
struct Layout {
    size_t scal, wp, head, clstart, clsize, cltoff, sched, queue, ctr, bar;
    size_t fl, fu1, fu2, fr, fpiv, u0n, tolv;
    size_t Y, T, partS, partG, partScal, vecS, vecX, vecR, qbuf, vbuf, tpub, gvec;
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
    kCtrCount = 8
};

struct Problem {
    int64_t n, m, ldz;
    const double* d;  // [n]
    const double* e;  // [n-1]
    const double* w;  // [m]
    double* Z;        // n x m, ldz
    int32_t* iters;   // [m] or null
    int32_t method;
    uint64_t seed;
    int64_t j0;
};

// All device pointers derived from one workspace (see Layout).
struct Ws {
    double* scal;     // [4]  onenrm, ortol, dtpcrt
    double* wp;       // [m]
    int32_t* head;    // [m]
    int32_t* clstart; // [m]
    int32_t* clsize;  // [m]
    int64_t* cltoff;  // [m]
    int32_t* sched;   // [P*4] team_first, team_size, team_rank, team_cluster
    int32_t* queue;   // [m]
    int64_t* ctr;     // [kCtrCount]
    uint32_t* bar;    // [P]
    double *fl, *fu1, *fu2, *fr;  // [m*n] LU factors, row j = shift j
    uint8_t* fpiv;    // [m*n]
    double* u0n;      // [m]   |u_nn| before perturbation
    double* tolv;     // [m]   tiny-pivot threshold eps max|U| per shift
    double* Y;        // [n*m]
    double* T;        // [m*m]
    double *partS, *partG;  // [P*n]
    double* partScal;       // [P*kScalTeam]
    double *vecS, *vecX, *vecR, *qbuf;  // [P*n]
    double* vbuf;     // [P*n]  solved iterate of each team (rows of all CTAs)
    double* tpub;     // [P*8]  published solve maps of each team (2 + 6 doubles per rank)
    double* gvec;     // [P*2n] global fallback for the per-CTA vectors (large n)
    int32_t P;        // persistent grid size the schedule was made for
    int32_t use_smem; // per-CTA vectors live in shared memory
};

Layout make_layout(int64_t n, int64_t m, int32_t P, bool need_chain);
Ws bind_layout(void* base, const Layout& L, int64_t n, int64_t m, int32_t P);

// Kernel launchers (tinv_kernels.cu).  All enqueue on `st` and return cudaGetLastError().
cudaError_t launch_plan(const Problem& p, const Ws& w, int32_t max_team, cudaStream_t st);
// LU of T - shift_j I for all j.  With tolv != null the diagonal is turned into perturbed
// reciprocals r = 1/u0 (solve-ready) and tolv[j] receives the tiny-pivot threshold; with
// tolv == null u0 is left as is.
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
cudaError_t launch_orth_plan(int64_t m, const Ws& w, int32_t method, cudaStream_t st);
cudaError_t launch_finish_info(const Problem& p, const Ws& w, int64_t* info_out, cudaStream_t st);

// Persistent-grid size (co-resident CTAs of the chain kernel) for order n on the current device,
// and the threads per CTA it runs with (256 with two CTAs per SM, or 512 with one).
int32_t chain_grid(int32_t cap, int64_t n);
int32_t chain_threads(int64_t n);
size_t chain_smem_bytes(int64_t n, bool use_smem);
bool chain_use_smem(int64_t n);

}  // namespace tinvx
