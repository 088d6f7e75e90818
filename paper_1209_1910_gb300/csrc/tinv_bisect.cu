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
                                                          int64_t n1, const double* __restrict__ D,
                                                          const double* __restrict__ E,
                                                          double* __restrict__ W)
{
    const int64_t q = blockIdx.y;
    const int64_t n = ns ? ns[q] : n1;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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

}  // namespace

// nprob problems; ns/offs are DEVICE arrays (or null for one problem of order n1 at offset 0).
cudaError_t launch_bisect(int64_t nprob, const int64_t* ns, const int64_t* offs, int64_t n1,
                          int64_t nmax, const double* d, const double* e, double* w, cudaStream_t st)
{
    if (nprob <= 0 || nmax <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((nmax + kBisectThreads - 1) / kBisectThreads), (unsigned)nprob);
    k_bisect<<<grid, kBisectThreads, 0, st>>>(ns, offs, n1, d, e, w);
    return cudaGetLastError();
}

}  // namespace tinvx

using namespace tinvx;

namespace {

int code_of(cudaError_t e)
{
    if (e == cudaSuccess) return TINV_OK;
    if (e == cudaErrorMemoryAllocation) return TINV_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
        e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDevice)
        return TINV_ENODEV;
    return TINV_ECUDA;
}

bool finite_all(const double* a, int64_t k)
{
    for (int64_t i = 0; i < k; ++i)
        if (!isfinite(a[i])) return false;
    return true;
}

}  // namespace

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
            if (!finite_all(d + off_de[q], n[q])) return -4;
            if (n[q] > 1 && !finite_all(e + off_de[q], n[q] - 1)) return -5;
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
    return code_of(ce);
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
