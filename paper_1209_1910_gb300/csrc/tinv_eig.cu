// tinv_eig.cu -- all eigenpairs of T with T split into unreduced blocks first (the IBLOCK/ISPLIT
// convention of DSTEIN, whose eigenvalues come from DSTEBZ; the paper's experiments take their
// eigenvalues the same way, Sec. 5.1).
//
// Row i ends a block iff |e_i| <= eps ||T||_1 (the paper is silent on the rule; dropping such an
// entry perturbs T by at most eps ||T||_1, within the residual bound of the method).  The blocks
// are independent problems: their eigenvalues come from the batched bisection, their
// eigenvectors from one tinv_batch launch sequence, and the results are merged into ascending
// order (ties keep the lower block first) and scattered into Z, zero outside each block.
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/tinv.h"
#include "tinv_internal.h"

namespace tinvx {
namespace {

constexpr int kSplitThreads = 1024;
constexpr int64_t kBisectChunk = 65535;  // problems per bisection launch (grid.y limit)



// ||T||_1 (max over rows of |d_i| + |e_{i-1}| + |e_i|, each row summed in that order; the
// maximum does not depend on the order of the rows) and the negligible entries: mark[i] = 1 iff
// |e_i| <= eps ||T||_1.  One CTA.
__global__ void __launch_bounds__(kSplitThreads) k_split(int64_t n, const double* __restrict__ d,
                                                         const double* __restrict__ e,
                                                         uint8_t* __restrict__ mark)
{
    __shared__ double s_red[kSplitThreads / 32];
    __shared__ double s_tol;
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double s = fabs(d[i]);
        if (i > 0) s = __dadd_rn(s, fabs(e[i - 1]));
        if (i < n - 1) s = __dadd_rn(s, fabs(e[i]));
        mx = fmax(mx, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_red[w]);
        s_tol = __dmul_rn(DBL_EPSILON, m);
    }
    __syncthreads();
    const double tol = s_tol;
    for (int64_t i = threadIdx.x; i < n - 1; i += blockDim.x) mark[i] = fabs(e[i]) <= tol ? 1 : 0;
}

// Column j of the merged result: source position src = perm[j] (the block-ordered position of
// the eigenvalue, which is also a row index), block b = blk[src]; rows of the block come from
// the block's packed eigenvector matrix, the other rows are zero.
__global__ void k_scatter(int64_t n, const int64_t* __restrict__ perm, const int32_t* __restrict__ blk,
                          const int64_t* __restrict__ bstart, const int64_t* __restrict__ bsize,
                          const int64_t* __restrict__ boffz, const double* __restrict__ wp,
                          const double* __restrict__ Zp, const int32_t* __restrict__ itp,
                          double* __restrict__ w, double* __restrict__ Z, int64_t ldz,
                          int64_t* __restrict__ iblock, int32_t* __restrict__ iters)
{
    const int64_t j = blockIdx.x;
    const int64_t src = perm[j];
    const int32_t b = blk[src];
    const int64_t s0 = bstart[b], nb = bsize[b], l = src - s0;
    const double* zc = Zp + boffz[b] + l * nb;
    double* dst = Z + j * ldz;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x)
        dst[r] = (r >= s0 && r < s0 + nb) ? zc[r - s0] : 0.0;
    if (threadIdx.x == 0) {
        w[j] = wp[src];
        if (iblock) iblock[j] = b;
        if (iters) iters[j] = itp[src];
    }
}

}  // namespace
}  // namespace tinvx

using namespace tinvx;

namespace {

// Block table from the split marks (host).
void blocks_from_marks(int64_t n, const uint8_t* mark, std::vector<int64_t>& start,
                       std::vector<int64_t>& size)
{
    start.clear();
    size.clear();
    int64_t b0 = 0;
    for (int64_t i = 0; i + 1 < n; ++i)
        if (mark[i]) {
            start.push_back(b0);
            size.push_back(i + 1 - b0);
            b0 = i + 1;
        }
    start.push_back(b0);
    size.push_back(n - b0);
}


// Split marks for device arrays d, e on stream st, returned in host memory.
int split_marks(int64_t n, const double* dd, const double* de, std::vector<uint8_t>& mark, cudaStream_t st)
{
    mark.assign((size_t)(n > 1 ? n - 1 : 1), 0);
    if (n <= 1) return 0;
    DevBuf m;
    cudaError_t ce = m.alloc((size_t)(n - 1), st, true);
    if (ce == cudaSuccess) {
        k_split<<<1, kSplitThreads, 0, st>>>(n, dd, de, (uint8_t*)m.p);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(mark.data(), m.p, (size_t)(n - 1), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    return cuda_code(ce);
}

}  // namespace

extern "C" int tinv_split(int64_t n, const double* d, const double* e, int64_t* isplit,
                          int64_t* nblock, const tinv_opts* o)
{
    tinv_opts op;
    if (o)
        op = *o;
    else
        tinv_opts_default(&op);
    if (n < 0) return -1;
    if (!nblock) return -5;
    if (n == 0) {
        *nblock = 0;
        return 0;
    }
    if (!d) return -2;
    if (n > 1 && !e) return -3;
    if (!isplit) return -4;
    if (!op.device_ptrs) {
        if (!all_finite(d, n)) return -2;
        if (n > 1 && !all_finite(e, n - 1)) return -3;
    }
    cudaStream_t st = nullptr;
    bool own = false;
    if (op.device_ptrs) {
        st = (cudaStream_t)op.stream;
    } else {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
        own = true;
    }
    int rc = 0;
    std::vector<uint8_t> mark;
    {
        DevBuf bd, be;
        const double *pd = d, *pe = e;
        if (!op.device_ptrs) {
            cudaError_t ce = bd.alloc((size_t)n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = be.alloc((size_t)(n > 1 ? n - 1 : 1) * sizeof(double), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(bd.p, d, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && n > 1)
                ce = cudaMemcpyAsync(be.p, e, (size_t)(n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            rc = cuda_code(ce);
            pd = (const double*)bd.p;
            pe = (const double*)be.p;
        }
        if (!rc) rc = split_marks(n, pd, pe, mark, st);
    }
    if (!rc) {
        std::vector<int64_t> start, size;
        blocks_from_marks(n, mark.data(), start, size);
        for (size_t b = 0; b < start.size(); ++b) isplit[b] = start[b] + size[b];
        *nblock = (int64_t)start.size();
    }
    if (own) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

extern "C" int tinv_eig(int64_t n, const double* d, const double* e, double* w, double* Z,
                        int64_t ldz, int64_t* iblock, int64_t* isplit, int64_t* nblock,
                        const tinv_opts* o)
{
    tinv_opts op;
    if (o)
        op = *o;
    else
        tinv_opts_default(&op);
    if (n < 0) return -1;
    if (op.method != TINV_CWY && op.method != TINV_MGS) return -10;
    if (n == 0) {
        if (nblock) *nblock = 0;
        return 0;
    }
    if (!d) return -2;
    if (n > 1 && !e) return -3;
    if (!w) return -4;
    if (!Z) return -5;
    if (ldz < n) return -6;
    if (!op.device_ptrs) {
        if (!all_finite(d, n)) return -2;
        if (n > 1 && !all_finite(e, n - 1)) return -3;
    }
    cudaStream_t st = nullptr;
    bool own = false;
    if (op.device_ptrs) {
        st = (cudaStream_t)op.stream;
    } else {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
        own = true;
    }
    int rc = 0;
    {
        const bool dev = op.device_ptrs != 0;
        DevBuf bd, be, bw, bz, bib, bit;
        const double *pd = d, *pe = e;
        double *pw = w, *pz = Z;
        int64_t* pib = iblock;
        int32_t* pit = op.iters;
        cudaError_t ce = cudaSuccess;
        if (!dev) {
            ce = bd.alloc((size_t)n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = be.alloc((size_t)(n > 1 ? n - 1 : 1) * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bw.alloc((size_t)n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bz.alloc((size_t)(n * ldz) * sizeof(double), st, true);
            if (ce == cudaSuccess && iblock) ce = bib.alloc((size_t)n * sizeof(int64_t), st, true);
            if (ce == cudaSuccess && op.iters) ce = bit.alloc((size_t)n * sizeof(int32_t), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(bd.p, d, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && n > 1)
                ce = cudaMemcpyAsync(be.p, e, (size_t)(n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            pd = (const double*)bd.p;
            pe = (const double*)be.p;
            pw = (double*)bw.p;
            pz = (double*)bz.p;
            pib = iblock ? (int64_t*)bib.p : nullptr;
            pit = op.iters ? (int32_t*)bit.p : nullptr;
        }
        rc = cuda_code(ce);
        // ---- blocks ----
        std::vector<uint8_t> mark;
        if (!rc) rc = split_marks(n, pd, pe, mark, st);
        std::vector<int64_t> start, size, offz;
        if (!rc) {
            blocks_from_marks(n, mark.data(), start, size);
            offz.resize(start.size());
            int64_t oz = 0;
            for (size_t b = 0; b < start.size(); ++b) {
                offz[b] = oz;
                oz += size[b] * size[b];
            }
            if (isplit)
                for (size_t b = 0; b < start.size(); ++b) isplit[b] = start[b] + size[b];
            if (nblock) *nblock = (int64_t)start.size();
        }
        const int64_t nb = (int64_t)start.size();
        int64_t zlen = 0, nmax = 0;
        for (int64_t b = 0; b < nb; ++b) {
            zlen += size[(size_t)b] * size[(size_t)b];
            nmax = std::max(nmax, size[(size_t)b]);
        }
        // ---- per-block eigenvalues (packed by row position) and eigenvectors (packed) ----
        DevBuf btab, bwp, bzp, bitp, binfo, bperm, bblk;
        if (!rc) {
            ce = btab.alloc((size_t)(3 * nb) * sizeof(int64_t), st, true);
            if (ce == cudaSuccess) ce = bwp.alloc((size_t)n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bzp.alloc((size_t)zlen * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bitp.alloc((size_t)n * sizeof(int32_t), st, true);
            if (ce == cudaSuccess) ce = binfo.alloc((size_t)nb * sizeof(int64_t), st, true);
            rc = cuda_code(ce);
        }
        std::vector<int64_t> tab;
        if (!rc) {
            tab.resize((size_t)(3 * nb));
            memcpy(tab.data(), size.data(), (size_t)nb * sizeof(int64_t));
            memcpy(tab.data() + nb, start.data(), (size_t)nb * sizeof(int64_t));
            memcpy(tab.data() + 2 * nb, offz.data(), (size_t)nb * sizeof(int64_t));
            ce = cudaMemcpyAsync(btab.p, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
            const int64_t* tn = (const int64_t*)btab.p;
            for (int64_t c0 = 0; c0 < nb && ce == cudaSuccess; c0 += kBisectChunk) {
                const int64_t cnt = std::min(kBisectChunk, nb - c0);
                int64_t cmax = 0;
                for (int64_t b = c0; b < c0 + cnt; ++b) cmax = std::max(cmax, size[(size_t)b]);
                ce = launch_bisect(cnt, tn + c0, tn + nb + c0, 0, cmax, pd, pe, (double*)bwp.p, st);
            }
            rc = cuda_code(ce);
        }
        if (!rc) {
            tinv_opts bo = op;
            bo.device_ptrs = 1;
            bo.stream = (void*)st;
            bo.workspace = nullptr;
            bo.workspace_bytes = 0;
            bo.iters = (int32_t*)bitp.p;
            bo.info = nullptr;
            bo.counters = nullptr;
            bo.table_ready = 0;
            rc = batch_enqueue_device(nb, size.data(), start.data(), offz.data(), nullptr, pd, pe,
                                      (const double*)bwp.p, (double*)bzp.p, (int64_t*)binfo.p, bo);
        }
        // ---- merge: stable order of the block eigenvalues (host), scatter (device) ----
        std::vector<double> wp;
        std::vector<int64_t> binf((size_t)nb);
        if (!rc) {
            wp.resize((size_t)n);
            ce = cudaMemcpyAsync(wp.data(), bwp.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(binf.data(), binfo.p, (size_t)nb * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
        std::vector<int64_t> perm;
        std::vector<int32_t> blk;
        if (!rc) {
            perm.resize((size_t)n);
            std::iota(perm.begin(), perm.end(), (int64_t)0);
            std::stable_sort(perm.begin(), perm.end(),
                             [&](int64_t a, int64_t b) { return wp[(size_t)a] < wp[(size_t)b]; });
            blk.resize((size_t)n);
            for (int64_t b = 0; b < nb; ++b)
                for (int64_t r = start[(size_t)b]; r < start[(size_t)b] + size[(size_t)b]; ++r)
                    blk[(size_t)r] = (int32_t)b;
            ce = bperm.alloc((size_t)n * sizeof(int64_t), st, true);
            if (ce == cudaSuccess) ce = bblk.alloc((size_t)n * sizeof(int32_t), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(bperm.p, perm.data(), (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(bblk.p, blk.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) {
                const int64_t* tn = (const int64_t*)btab.p;
                k_scatter<<<(unsigned)n, 256, 0, st>>>(n, (const int64_t*)bperm.p, (const int32_t*)bblk.p,
                                                      tn + nb, tn, tn + 2 * nb, (const double*)bwp.p,
                                                      (const double*)bzp.p, (const int32_t*)bitp.p, pw, pz,
                                                      ldz, pib, pit);
                ce = cudaGetLastError();
            }
            if (ce == cudaSuccess && !dev) {
                ce = cudaMemcpyAsync(w, pw, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpy2DAsync(Z, (size_t)ldz * sizeof(double), pz, (size_t)ldz * sizeof(double),
                                           (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToHost, st);
                if (ce == cudaSuccess && iblock)
                    ce = cudaMemcpyAsync(iblock, pib, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
                if (ce == cudaSuccess && op.iters)
                    ce = cudaMemcpyAsync(op.iters, pit, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            }
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
        if (!rc) {
            int64_t cnt = 0;
            bool timed_out = false;
            for (int64_t b = 0; b < nb; ++b) {
                if (binf[(size_t)b] == TINV_ETIMEDOUT) timed_out = true;
                else cnt += binf[(size_t)b];
            }
            rc = timed_out ? TINV_ETIMEDOUT : (cnt > INT32_MAX ? INT32_MAX : (int)cnt);
        }
    }
    if (own) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}
