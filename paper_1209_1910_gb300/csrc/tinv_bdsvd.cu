// tinv_bdsvd.cu -- singular triplets of an upper bidiagonal B (diagonal a[n], superdiagonal
// b[n-1]) by the inverse iteration of this library applied to B's Golub-Kahan form (the paper's
// Sec. 6 names singular vectors of a bidiagonal matrix as a further use of the method).
//
// T_GK is the symmetric tridiagonal matrix of order 2n with zero diagonal and off-diagonal
// (a_1, b_1, a_2, b_2, ..., a_n); its eigenvalues are +-sigma_i, and the eigenvector of +sigma
// interleaves v and u: (v_1, u_1, ..., v_n, u_n) / sqrt(2) with B v = sigma u, B^T u = sigma v.
// The eigenvector of -sigma is the same with u negated, so a computed vector that mixes the two
// still has its even entries along v and its odd entries along u: each half is scaled to unit
// length on its own.
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/tinv.h"
#include "tinv_internal.h"

namespace tinvx {
namespace {

constexpr int kSplitHalfThreads = 256;



// T_GK: d2 = 0 (2n), e2 = (a_1, b_1, ..., a_n) (2n - 1).
__global__ void k_golub_kahan(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ d2, double* __restrict__ e2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        d2[i] = 0.0;
        if (i < 2 * n - 1) e2[i] = (i & 1) ? b[i >> 1] : a[i >> 1];
    }
}

// Column j of Z2 (2n rows): v = even rows, u = odd rows, each scaled to unit 2-norm (the sum of
// squares is added by a fixed-shape reduction; a half that is all zero stays zero).
__global__ void __launch_bounds__(kSplitHalfThreads) k_split_halves(int64_t n, const double* __restrict__ Z2,
                                                                    double* __restrict__ U, int64_t ldu,
                                                                    double* __restrict__ V, int64_t ldv)
{
    __shared__ double s_v[kSplitHalfThreads / 32], s_u[kSplitHalfThreads / 32];
    __shared__ double s_nrm[2];
    const int64_t j = blockIdx.x;
    const double* z = Z2 + j * 2 * n;
    double sv = 0.0, su = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = z[2 * i], u = z[2 * i + 1];
        sv = fma(v, v, sv);
        su = fma(u, u, su);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
        su += __shfl_xor_sync(0xffffffffu, su, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_v[threadIdx.x >> 5] = sv;
        s_u[threadIdx.x >> 5] = su;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tv = 0.0, tu = 0.0;
        for (int w = 0; w < kSplitHalfThreads / 32; ++w) {
            tv += s_v[w];
            tu += s_u[w];
        }
        s_nrm[0] = sqrt(tv);
        s_nrm[1] = sqrt(tu);
    }
    __syncthreads();
    const double nv = s_nrm[0], nu = s_nrm[1];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = z[2 * i], u = z[2 * i + 1];
        V[i + j * ldv] = nv > 0.0 ? v / nv : 0.0;
        U[i + j * ldu] = nu > 0.0 ? u / nu : 0.0;
    }
}


}  // namespace
}  // namespace tinvx

using namespace tinvx;

extern "C" int tinv_bdsvd(int64_t n, const double* a, const double* b, double* s, double* U,
                          int64_t ldu, double* V, int64_t ldv, const tinv_opts* o)
{
    tinv_opts op;
    if (o)
        op = *o;
    else
        tinv_opts_default(&op);
    if (n < 0) return -1;
    if (op.method != TINV_CWY && op.method != TINV_MGS) return -9;
    if (n == 0) return 0;
    if (!a) return -2;
    if (n > 1 && !b) return -3;
    if (!s) return -4;
    if (!U) return -5;
    if (ldu < n) return -6;
    if (!V) return -7;
    if (ldv < n) return -8;
    if (n > (int64_t)INT32_MAX / 4) return TINV_ENOTSUP;
    if (!op.device_ptrs) {
        if (!all_finite(a, n)) return -2;
        if (n > 1 && !all_finite(b, n - 1)) return -3;
    }
    cudaStream_t st = nullptr;
    bool own = false;
    if (op.device_ptrs) {
        st = (cudaStream_t)op.stream;
    } else {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
        own = true;
    }
    const bool dev = op.device_ptrs != 0;
    const int64_t n2 = 2 * n;
    int rc = 0;
    {
        DevBuf ba, bb, bu, bv, bd2, be2, bw2, bz2, binfo, bit;
        const double *pa = a, *pb = b;
        double *pu = U, *pv = V;
        cudaError_t ce = cudaSuccess;
        if (!dev) {
            ce = ba.alloc((size_t)n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bb.alloc((size_t)(n > 1 ? n - 1 : 1) * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bu.alloc((size_t)(n * ldu) * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bv.alloc((size_t)(n * ldv) * sizeof(double), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(ba.p, a, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && n > 1)
                ce = cudaMemcpyAsync(bb.p, b, (size_t)(n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            pa = (const double*)ba.p;
            pb = (const double*)bb.p;
            pu = (double*)bu.p;
            pv = (double*)bv.p;
        }
        if (ce == cudaSuccess) ce = bd2.alloc((size_t)n2 * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = be2.alloc((size_t)(n2 - 1) * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = bw2.alloc((size_t)n2 * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = bz2.alloc((size_t)(n2 * n) * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = binfo.alloc(sizeof(int64_t), st, true);
        if (ce == cudaSuccess && op.iters && !dev) ce = bit.alloc((size_t)n * sizeof(int32_t), st, true);
        if (ce == cudaSuccess) {
            const unsigned g = (unsigned)((n2 + 255) / 256 < 4096 ? (n2 + 255) / 256 : 4096);
            k_golub_kahan<<<g, 256, 0, st>>>(n, pa, pb, (double*)bd2.p, (double*)be2.p);
            ce = cudaGetLastError();
        }
        // the n largest of the 2n eigenvalues by bisection (indices n .. 2n-1, into bw2 + n):
        // the singular values, ascending
        if (ce == cudaSuccess)
            ce = launch_bisect(1, nullptr, nullptr, n2, n2, (const double*)bd2.p, (const double*)be2.p,
                               (double*)bw2.p, st, n);
        rc = cuda_code(ce);
        if (!rc) {
            tinv_opts to = op;
            to.device_ptrs = 1;
            to.stream = (void*)st;
            to.info = (int64_t*)binfo.p;
            to.iters = op.iters ? (dev ? op.iters : (int32_t*)bit.p) : nullptr;
            to.counters = nullptr;
            to.workspace = nullptr;
            to.workspace_bytes = 0;
            rc = tinv_ex(n2, (const double*)bd2.p, (const double*)be2.p, n, (const double*)bw2.p + n,
                         (double*)bz2.p, n2, &to, nullptr);
        }
        if (!rc) {
            k_split_halves<<<(unsigned)n, kSplitHalfThreads, 0, st>>>(n, (const double*)bz2.p, pu, ldu, pv, ldv);
            ce = cudaGetLastError();
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(s, (const double*)bw2.p + n, (size_t)n * sizeof(double),
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess && !dev) {
                // the caller's rows n .. ld-1 of each column are left untouched
                ce = cudaMemcpy2DAsync(U, (size_t)ldu * sizeof(double), pu, (size_t)ldu * sizeof(double),
                                       (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToHost, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpy2DAsync(V, (size_t)ldv * sizeof(double), pv, (size_t)ldv * sizeof(double),
                                           (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToHost, st);
                if (ce == cudaSuccess && op.iters)
                    ce = cudaMemcpyAsync(op.iters, bit.p, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            }
            int64_t info = 0;
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(&info, binfo.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
            if (!rc) rc = info > INT32_MAX ? INT32_MAX : (int)info;
        }
    }
    if (own) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}
