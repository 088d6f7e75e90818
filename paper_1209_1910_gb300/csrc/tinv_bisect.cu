// tinv_bisect.cu -- eigenvalue approximations by Sturm-count bisection on the GPU: the step
// before inverse iteration (the paper obtains its eigenvalues with LAPACK's bisection, Sec. 5.1).
//
// One thread per eigenvalue (all problems of a batch in one launch: blockIdx.y is the problem,
// blockIdx.x * blockDim.x + threadIdx.x the eigenvalue index k).  Eigenvalue k is bracketed in the
// widened Gershgorin interval and halved until the bracket is below
// max(2 eps max(|lo|, |hi|), eps ||T||_1); the count of eigenvalues below x is the number of
// negative pivots q_i of the LDL^T factorization of T - x I, with pivots smaller than
// pivmin = DBL_MIN max(1, max e_i^2) in magnitude replaced by -pivmin.  Every operation is an
// explicit round-to-nearest FP64 operation (no contraction), evaluated in the order of a plain
// sequential loop, so the result does not depend on the launch shape.
#include <float.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/tinv.h"
#include "tinv_internal.h"

namespace tinvx {
namespace {

constexpr double kEpsB = 2.220446049250313080847e-16;  // 2^-52
constexpr int kBisectThreads = 128;
constexpr int kMaxBisect = 4000;  // bound on halvings (about 2100 reach the smallest subnormal)

__device__ __forceinline__ double dmax_(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double dmin_(double a, double b) { return a < b ? a : b; }

// Number of eigenvalues of T smaller than x.
__device__ __forceinline__ int64_t sturm_count(int64_t n, const double* __restrict__ d,
                                               const double* __restrict__ e, double x, double pivmin)
{
    int64_t cnt = 0;
    double q = __dsub_rn(d[0], x);
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
    for (int64_t i = 1; i < n; ++i) {
        const double ei = e[i - 1];
        q = __dsub_rn(__dsub_rn(d[i], x), __ddiv_rn(__dmul_rn(ei, ei), q));
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

__global__ void __launch_bounds__(kBisectThreads) k_bisect(const int64_t* __restrict__ ns,
                                                          const int64_t* __restrict__ offs,
                                                          int64_t n1, int64_t k0,
                                                          const double* __restrict__ D,
                                                          const double* __restrict__ E,
                                                          double* __restrict__ W)
{
    const int64_t q = blockIdx.y;
    const int64_t n = ns ? ns[q] : n1;
    const int64_t k = k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t off = offs ? offs[q] : 0;
    const double* d = D + off;
    const double* e = E + off;
    // Gershgorin interval, pivmin and ||T||_1, scanned in index order
    double glo = INFINITY, ghi = -INFINITY, emax2 = 0.0, onenrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = 0.0;
        if (i > 0) r = __dadd_rn(r, fabs(e[i - 1]));
        if (i < n - 1) {
            r = __dadd_rn(r, fabs(e[i]));
            emax2 = dmax_(emax2, __dmul_rn(e[i], e[i]));
        }
        glo = dmin_(glo, __dsub_rn(d[i], r));
        ghi = dmax_(ghi, __dadd_rn(d[i], r));
        double s = fabs(d[i]);
        if (i > 0) s = __dadd_rn(s, fabs(e[i - 1]));
        if (i < n - 1) s = __dadd_rn(s, fabs(e[i]));
        onenrm = dmax_(onenrm, s);
    }
    const double pivmin = __dmul_rn(DBL_MIN, dmax_(1.0, emax2));
    const double bnd = dmax_(fabs(glo), fabs(ghi));
    const double widen = __dadd_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, kEpsB), bnd), (double)n),
                                   __dmul_rn(2.0, pivmin));
    double lo = __dsub_rn(glo, widen), hi = __dadd_rn(ghi, widen);
    const double tol_abs = __dmul_rn(kEpsB, onenrm);
    for (int it = 0; it < kMaxBisect; ++it) {
        const double tol = dmax_(__dmul_rn(__dmul_rn(2.0, kEpsB), dmax_(fabs(lo), fabs(hi))), tol_abs);
        if (__dsub_rn(hi, lo) <= tol) break;
        const double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(n, d, e, mid, pivmin) <= k)
            lo = mid;
        else
            hi = mid;
    }
    W[off + k] = __dmul_rn(0.5, __dadd_rn(lo, hi));
}

// The same bisection with L = 2^S lanes per eigenvalue, for launches with too few eigenvalues to
// fill the GPU.  The next S halvings of the bracket can only visit the 2^S - 1 midpoints of a
// binary tree (node j's children bisect its two halves); lane j < L - 1 computes node j's
// midpoint by the same rounding formula along its path from the current bracket and the Sturm
// count there, all lanes in parallel.  The group then takes the S steps exactly as k_bisect
// does (same termination tests in the same order, the count of the node it reaches), so the
// result is bit-identical to k_bisect's; only the counts of nodes off the path are wasted.
template <int L>
__global__ void __launch_bounds__(kBisectThreads) k_bisect_tree(const int64_t* __restrict__ ns,
                                                               const int64_t* __restrict__ offs,
                                                               int64_t n1, int64_t k0,
                                                               const double* __restrict__ D,
                                                               const double* __restrict__ E,
                                                               double* __restrict__ W)
{
    constexpr int S = (L == 4) ? 2 : (L == 8) ? 3 : (L == 16) ? 4 : 5;
    const int64_t q = blockIdx.y;
    const int64_t n = ns ? ns[q] : n1;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = k0 + gt / L;  // the whole group of L lanes shares k
    const int g = (int)(gt % L);
    if (k >= n) return;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1)));
    const int64_t off = offs ? offs[q] : 0;
    const double* d = D + off;
    const double* e = E + off;
    double glo = INFINITY, ghi = -INFINITY, emax2 = 0.0, onenrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = 0.0;
        if (i > 0) r = __dadd_rn(r, fabs(e[i - 1]));
        if (i < n - 1) {
            r = __dadd_rn(r, fabs(e[i]));
            emax2 = dmax_(emax2, __dmul_rn(e[i], e[i]));
        }
        glo = dmin_(glo, __dsub_rn(d[i], r));
        ghi = dmax_(ghi, __dadd_rn(d[i], r));
        double sabs = fabs(d[i]);
        if (i > 0) sabs = __dadd_rn(sabs, fabs(e[i - 1]));
        if (i < n - 1) sabs = __dadd_rn(sabs, fabs(e[i]));
        onenrm = dmax_(onenrm, sabs);
    }
    const double pivmin = __dmul_rn(DBL_MIN, dmax_(1.0, emax2));
    const double bnd = dmax_(fabs(glo), fabs(ghi));
    const double widen = __dadd_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, kEpsB), bnd), (double)n),
                                   __dmul_rn(2.0, pivmin));
    double lo = __dsub_rn(glo, widen), hi = __dadd_rn(ghi, widen);
    const double tol_abs = __dmul_rn(kEpsB, onenrm);
    int it = 0;
    for (;;) {
        // node g of the tree: follow the bits of g + 1 below its leading one (0 = left half)
        int64_t cnt = 0;
        if (g < L - 1) {
            const unsigned path = (unsigned)g + 1u;
            const int depth = 31 - __clz(path);
            double blo = lo, bhi = hi;
            for (int dd = depth - 1; dd >= 0; --dd) {
                const double m = __dmul_rn(0.5, __dadd_rn(blo, bhi));
                if ((path >> dd) & 1u)
                    blo = m;
                else
                    bhi = m;
            }
            cnt = sturm_count(n, d, e, __dmul_rn(0.5, __dadd_rn(blo, bhi)), pivmin);
        }
        // the S steps of the sequential bisection, with the counts of the nodes on its path
        bool done = false;
        int j = 0;
        for (int lev = 0; lev < S; ++lev) {
            if (it >= kMaxBisect) {
                done = true;
                break;
            }
            const double tol = dmax_(__dmul_rn(__dmul_rn(2.0, kEpsB), dmax_(fabs(lo), fabs(hi))), tol_abs);
            if (__dsub_rn(hi, lo) <= tol) {
                done = true;
                break;
            }
            const double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
            if (mid <= lo || mid >= hi) {
                done = true;
                break;
            }
            const long long cj = __shfl_sync(gmask, (long long)cnt, j, L);
            if (cj <= k) {
                lo = mid;
                j = 2 * j + 2;
            } else {
                hi = mid;
                j = 2 * j + 1;
            }
            ++it;
        }
        if (done) break;
    }
    if (g == 0) W[off + k] = __dmul_rn(0.5, __dadd_rn(lo, hi));
}

}  // namespace

// Lanes per eigenvalue for a launch of nprob x neig eigenvalues: the largest of 32, 16, 8, 4 that
// keeps the launch within about one warp per SM sub-partition, else 1 (plain bisection).  One
// warp's FP64 instruction holds its sub-partition's FP64 pipe for about 64 cycles, so a single
// warp of dependent Sturm steps already keeps that pipe busy; more lanes then only add the tree's
// extra midpoints (2^S - 1 counts for S halvings).
int bisect_lanes(int64_t nprob, int64_t neig)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t target = (int64_t)(sms > 0 ? sms : 1) * 4 * 32;
    const int64_t eig = nprob * neig;
    for (int L = 32; L >= 4; L >>= 1)
        if (eig * L <= target) return L;
    return 1;
}

// nprob problems; ns/offs are DEVICE arrays (or null for one problem of order n1 at offset 0).
// Eigenvalues k0 .. n-1 of each problem are computed (k0 > 0 only for a single problem).
cudaError_t launch_bisect(int64_t nprob, const int64_t* ns, const int64_t* offs, int64_t n1,
                          int64_t nmax, const double* d, const double* e, double* w, cudaStream_t st,
                          int64_t k0)
{
    if (k0 < 0 || (k0 > 0 && ns)) return cudaErrorInvalidValue;
    const int64_t neig = nmax - k0;
    if (nprob <= 0 || neig <= 0) return cudaSuccess;
    const int L = bisect_lanes(nprob, neig);
    const dim3 grid((unsigned)((neig * L + kBisectThreads - 1) / kBisectThreads), (unsigned)nprob);
    switch (L) {
    case 32: k_bisect_tree<32><<<grid, kBisectThreads, 0, st>>>(ns, offs, n1, k0, d, e, w); break;
    case 16: k_bisect_tree<16><<<grid, kBisectThreads, 0, st>>>(ns, offs, n1, k0, d, e, w); break;
    case 8: k_bisect_tree<8><<<grid, kBisectThreads, 0, st>>>(ns, offs, n1, k0, d, e, w); break;
    case 4: k_bisect_tree<4><<<grid, kBisectThreads, 0, st>>>(ns, offs, n1, k0, d, e, w); break;
    default: k_bisect<<<grid, kBisectThreads, 0, st>>>(ns, offs, n1, k0, d, e, w); break;
    }
    return cudaGetLastError();
}

}  // namespace tinvx

using namespace tinvx;

extern "C" int tinv_bisect_batch(int64_t nprob, const int64_t* n, const int64_t* off_de,
                                 const double* d, const double* e, double* w, const tinv_opts* o)
{
    tinv_opts op;
    if (o)
        op = *o;
    else
        tinv_opts_default(&op);
    if (nprob < 0) return -1;
    if (nprob == 0) return 0;
    if (!n) return -2;
    if (!off_de) return -3;
    if (nprob > 65535) return TINV_ENOTSUP;
    int64_t nmax = 0, de_len = 0, e_len = 0;
    for (int64_t q = 0; q < nprob; ++q) {
        if (n[q] < 0) return -2;
        if (off_de[q] < 0) return -3;
        if (n[q] == 0) continue;
        nmax = n[q] > nmax ? n[q] : nmax;
        de_len = off_de[q] + n[q] > de_len ? off_de[q] + n[q] : de_len;
        e_len = off_de[q] + n[q] - 1 > e_len ? off_de[q] + n[q] - 1 : e_len;
    }
    if (nmax == 0) return 0;
    if (!d) return -4;
    if (e_len > 0 && !e) return -5;
    if (!w) return -6;
    if (!op.device_ptrs) {
        for (int64_t q = 0; q < nprob; ++q) {
            if (n[q] == 0) continue;
            if (!all_finite(d + off_de[q], n[q])) return -4;
            if (n[q] > 1 && !all_finite(e + off_de[q], n[q] - 1)) return -5;
        }
    }
    cudaStream_t st = nullptr;
    bool own = false;
    if (op.device_ptrs) {
        st = (cudaStream_t)op.stream;
    } else {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
        own = true;
    }
    // device copies: the problem table always, the arrays with host pointers
    void* tab = nullptr;
    double *dd = nullptr, *de = nullptr, *dw = nullptr;
    cudaError_t ce = cudaMallocAsync(&tab, (size_t)nprob * 2 * sizeof(int64_t), st);
    if (ce == cudaSuccess) {
        std::vector<int64_t> h((size_t)nprob * 2);
        memcpy(h.data(), n, (size_t)nprob * sizeof(int64_t));
        memcpy(h.data() + nprob, off_de, (size_t)nprob * sizeof(int64_t));
        ce = cudaMemcpyAsync(tab, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess && own) ce = cudaStreamSynchronize(st);
    }
    const double *pd = d, *pe = e;
    double* pw = w;
    if (ce == cudaSuccess && !op.device_ptrs) {
        ce = cudaMallocAsync((void**)&dd, (size_t)de_len * sizeof(double), st);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&de, (size_t)(e_len > 0 ? e_len : 1) * sizeof(double), st);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&dw, (size_t)de_len * sizeof(double), st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(dd, d, (size_t)de_len * sizeof(double), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess && e_len > 0)
            ce = cudaMemcpyAsync(de, e, (size_t)e_len * sizeof(double), cudaMemcpyHostToDevice, st);
        pd = dd;
        pe = de;
        pw = dw;
    }
    if (ce == cudaSuccess) {
        const int64_t* tn = (const int64_t*)tab;
        ce = launch_bisect(nprob, tn, tn + nprob, 0, nmax, pd, pe, pw, st);
    }
    if (ce == cudaSuccess && !op.device_ptrs) {
        for (int64_t q = 0; q < nprob && ce == cudaSuccess; ++q)
            if (n[q] > 0)
                ce = cudaMemcpyAsync(w + off_de[q], dw + off_de[q], (size_t)n[q] * sizeof(double),
                                     cudaMemcpyDeviceToHost, st);
    }
    if (tab) cudaFreeAsync(tab, st);
    if (dd) cudaFreeAsync(dd, st);
    if (de) cudaFreeAsync(de, st);
    if (dw) cudaFreeAsync(dw, st);
    if (own) {
        const cudaError_t s2 = cudaStreamSynchronize(st);
        if (ce == cudaSuccess) ce = s2;
        cudaStreamDestroy(st);
    }
    return cuda_code(ce);
}

extern "C" int tinv_bisect(int64_t n, const double* d, const double* e, double* w, const tinv_opts* o)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!d) return -2;
    if (n > 1 && !e) return -3;
    if (!w) return -4;
    const int64_t off = 0;
    const int rc = tinv_bisect_batch(1, &n, &off, d, e, w, o);
    // map the batch call's argument positions (d = 4, e = 5, w = 6) to this call's
    if (rc == -4) return -2;
    if (rc == -5) return -3;
    if (rc == -6) return -4;
    return rc;
}
