// tinv_api.cu -- host side of libtinv: argument checks, workspace layout, transfers and the
// launch sequence of the C ABI declared in include/tinv.h.
//
// Launch sequence of tinv_ex (one stream, no host synchronization in between):
//   k_plan (1 CTA)        a1-a2: ||T||_1, tolerances, perturbed shifts, clusters, team schedule
//   k_lu   (thread/shift) a3   : LU with scaled partial pivoting of T - w'_j I, all j
//   k_first(warp/shift)   a4-a5, a7-a8 for cluster heads and singletons; first sweep of members
//   k_chain(cooperative)  a5-a8 with a6 (compact WY or MGS) for cluster members, in order
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "../../include/tinv.h"
#include "tinv_internal.h"

namespace tinvx {

// One pool per (device, context): a pool belongs to the context it was created in (a driver
// context the caller made current, or a primary context re-created after cudaDeviceReset, has
// its own), so the cache is keyed by the unique id of the current context.
using PoolCtxGetCurrentFn = CUresult (*)(CUcontext*);
using PoolCtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
struct PoolEntry {
    unsigned long long ctx_id;
    cudaMemPool_t pool;
};
static std::mutex g_pool_mu;
static PoolEntry g_pools[64];
static int g_pool_used = 0;
static bool g_pool_fn_init = false;
static PoolCtxGetCurrentFn g_pool_ctx_cur = nullptr;
static PoolCtxGetIdFn g_pool_ctx_id = nullptr;

cudaMemPool_t lib_pool(cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    // a stream being captured into a graph takes a pool that exists; none is created then
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_fn_init) {
        g_pool_fn_init = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_pool_ctx_cur = (PoolCtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_pool_ctx_id = (PoolCtxGetIdFn)f;
    }
    if (!g_pool_ctx_cur || !g_pool_ctx_id) return nullptr;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_pool_ctx_cur(&ctx) != CUDA_SUCCESS || !ctx || g_pool_ctx_id(ctx, &id) != CUDA_SUCCESS)
        return nullptr;
    for (int i = 0; i < g_pool_used; ++i)
        if (g_pools[i].ctx_id == id) return g_pools[i].pool;
    if (g_pool_used == 64 || cap != cudaStreamCaptureStatusNone) return nullptr;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return nullptr;
    }
    g_pools[g_pool_used++] = {id, pool};
    return pool;
}

size_t lib_pool_idle()
{
    cudaMemPool_t pool = lib_pool(nullptr);
    if (!pool) return 0;
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess)
        return 0;
    return reserved > used ? (size_t)(reserved - used) : 0;
}


static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Dims single_dims(int64_t n, int64_t m, int32_t P, int32_t block)
{
    Dims D;
    D.nmax = n;
    D.M = m;
    D.F = n * m;
    D.TT = m * m;
    D.nseg = 1;
    D.P = P;
    D.block = block;
    return D;
}

int32_t opts_block(const tinv_opts& o)
{
    if (o.method != TINV_CWY || o.block <= 1) return 0;
    return o.block < kBlockMax ? o.block : kBlockMax;
}

Layout make_layout(const Dims& D, bool need_chain, bool need_rhs)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return o;
    };
    const size_t nn = (size_t)D.nmax, mm = (size_t)D.M, ff = (size_t)D.F, pp = (size_t)D.P;
    L.segs = take((size_t)D.nseg * sizeof(Seg));
    L.segj = take(mm * sizeof(int32_t));
    L.sinfo = take((size_t)D.nseg * sizeof(int64_t));
    L.scal = take(4 * sizeof(double));
    L.wp = take(mm * sizeof(double));
    L.head = take(mm * sizeof(int32_t));
    L.clstart = take(mm * sizeof(int32_t));
    L.clsize = take(mm * sizeof(int32_t));
    L.cltoff = take(mm * sizeof(int64_t));
    L.sched = take(pp * 4 * sizeof(int32_t));
    L.queue = take(mm * sizeof(int32_t));
    L.ctr = take(kCtrCount * sizeof(int64_t));
    L.bar = take(pp * sizeof(uint32_t));
    L.fl = take(ff * sizeof(double));
    L.fu1 = take(ff * sizeof(double));
    L.fu2 = take(ff * sizeof(double));
    L.fr = take(ff * sizeof(double));
    L.fpiv = take(ff);
    L.u0n = take(mm * sizeof(double));
    L.tolv = take(mm * sizeof(double));
    if (need_rhs) L.rhs = take(ff * sizeof(double));
    if (need_chain) {
        L.Y = take(ff * sizeof(double));
        L.T = take((size_t)D.TT * sizeof(double));
        L.partS = take(pp * nn * sizeof(double));
        L.partG = take(pp * nn * sizeof(double));
        L.partScal = take(pp * kScalTeam * sizeof(double));
        L.vecS = take(pp * nn * sizeof(double));
        L.vecX = take(pp * nn * sizeof(double));
        L.vecR = take(pp * nn * sizeof(double));
        L.qbuf = take(pp * nn * sizeof(double));
        L.vbuf = take(pp * nn * sizeof(double));
        L.tpub = take(pp * 8 * sizeof(double));
        if (!chain_use_smem(D.nmax)) L.gvec = take(pp * 2 * nn * sizeof(double));
        if (D.block >= 2 && block_xcap(D.nmax) > 0) {
            const size_t bv = pp * (size_t)kBlockMax * nn * sizeof(double);
            L.vblk = take(bv);
            L.qblk = take(bv);
            L.pblk = take(3 * bv);
            L.tblk = take(3 * bv);
        }
    }
    L.total = off;
    return L;
}

Ws bind_layout(void* base, const Layout& L, const Dims& D)
{
    char* b = (char*)base;
    Ws w;
    memset(&w, 0, sizeof(w));
    w.segs = (Seg*)(b + L.segs);
    w.segj = (int32_t*)(b + L.segj);
    w.sinfo = (int64_t*)(b + L.sinfo);
    w.scal = (double*)(b + L.scal);
    w.wp = (double*)(b + L.wp);
    w.head = (int32_t*)(b + L.head);
    w.clstart = (int32_t*)(b + L.clstart);
    w.clsize = (int32_t*)(b + L.clsize);
    w.cltoff = (int64_t*)(b + L.cltoff);
    w.sched = (int32_t*)(b + L.sched);
    w.queue = (int32_t*)(b + L.queue);
    w.ctr = (int64_t*)(b + L.ctr);
    w.bar = (uint32_t*)(b + L.bar);
    w.fl = (double*)(b + L.fl);
    w.fu1 = (double*)(b + L.fu1);
    w.fu2 = (double*)(b + L.fu2);
    w.fr = (double*)(b + L.fr);
    w.fpiv = (uint8_t*)(b + L.fpiv);
    w.u0n = (double*)(b + L.u0n);
    w.tolv = (double*)(b + L.tolv);
    w.rhs = L.rhs ? (double*)(b + L.rhs) : nullptr;
    if (L.Y) {
        w.Y = (double*)(b + L.Y);
        w.T = (double*)(b + L.T);
        w.partS = (double*)(b + L.partS);
        w.partG = (double*)(b + L.partG);
        w.partScal = (double*)(b + L.partScal);
        w.vecS = (double*)(b + L.vecS);
        w.vecX = (double*)(b + L.vecX);
        w.vecR = (double*)(b + L.vecR);
        w.qbuf = (double*)(b + L.qbuf);
        w.vbuf = (double*)(b + L.vbuf);
        w.tpub = (double*)(b + L.tpub);
        w.gvec = L.gvec ? (double*)(b + L.gvec) : nullptr;
        if (L.vblk) {
            w.vblk = (double*)(b + L.vblk);
            w.qblk = (double*)(b + L.qblk);
            w.pblk = (double*)(b + L.pblk);
            w.tblk = (double*)(b + L.tblk);
            w.block = D.block;
            w.xcap = block_xcap(D.nmax);
        }
    }
    w.P = D.P;
    w.use_smem = chain_use_smem(D.nmax) ? 1 : 0;
    w.nF = D.F;
    w.nTT = D.TT;
    w.nM = D.M;
    w.nPN = (int64_t)D.P * D.nmax;
#ifdef TINV_DEBUG
    // test hook of the debug build: declare Y shorter than it is (by this many elements), so
    // the bounds checks of the cluster kernel must fire on accesses that are still inside the
    // real allocation (the check skips them)
    if (const char* sh = getenv("TINV_DEBUG_SHRINK_F")) {
        const long long k = atoll(sh);
        if (k > 0) w.nF = w.nF > k ? w.nF - k : 0;
    }
#endif
    return w;
}

}  // namespace tinvx

using namespace tinvx;

namespace {

__device__ __forceinline__ int64_t dev_err_code(int64_t err)
{
    if (err & kErrBounds) return TINV_EINTERNAL;
    return err ? (int64_t)TINV_ETIMEDOUT : 0;
}

__global__ void k_finish(const int64_t* ctr, int64_t* info)
{
    const int64_t err = ctr[kCtrErr];
    *info = err ? dev_err_code(err) : ctr[kCtrInfo];
}

// tinv_opts.counters from the counter block.
__global__ void k_counters(const int64_t* ctr, int64_t* out)
{
    out[0] = ctr[kCtrFallback];
    out[1] = ctr[kCtrNClust];
    out[2] = ctr[kCtrNClust] - ctr[kCtrNQueue];
    out[3] = ctr[kCtrFallbackFirst];
}

void host_counters(const int64_t* ctr, int64_t* out)
{
    out[0] = ctr[kCtrFallback];
    out[1] = ctr[kCtrNClust];
    out[2] = ctr[kCtrNClust] - ctr[kCtrNQueue];
    out[3] = ctr[kCtrFallbackFirst];
}

// Per-problem results of a batch: the non-converged count, or the timeout code for all.
__global__ void k_finish_batch(const int64_t* ctr, const int64_t* sinfo, int64_t nprob, int64_t* info)
{
    const int64_t err = ctr[kCtrErr];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nprob;
         q += (int64_t)gridDim.x * blockDim.x)
        info[q] = err ? dev_err_code(err) : sinfo[q];
}

struct Opts {
    tinv_opts o;
    explicit Opts(const tinv_opts* src)
    {
        if (src)
            o = *src;
        else
            tinv_opts_default(&o);
    }
};

// Enqueue the full inverse-iteration path on `st` for problems whose arrays are all on the
// device.  `ws` must hold make_layout(D, true).total bytes; with p.seg_preset the problem table
// must already be in the workspace (copied on `st`).
// When phase_ms is given, CUDA events bracket each launch and the elapsed device times are
// stored after synchronizing on the last event.
int enqueue_tinv(const Problem& p0, void* ws, const Dims& D, int32_t max_team, cudaStream_t st,
                 float* phase_ms)
{
    const Layout L = make_layout(D, true);
    const Ws w = bind_layout(ws, L, D);
    Problem p = p0;
    if (!p.seg_preset && p.zlen == 0 && p.m > 0) p.zlen = (p.m - 1) * p.ldz + p.n;
    cudaEvent_t ev[5] = {};
    cudaError_t e = cudaSuccess;
    if (phase_ms) {
        for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    }
    if (e == cudaSuccess) e = launch_plan(p, w, max_team, st);
    if (e == cudaSuccess && phase_ms) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = launch_lu_seg(p, w, st);
    if (e == cudaSuccess && phase_ms) e = cudaEventRecord(ev[2], st);
    if (e == cudaSuccess) e = launch_first(p, w, st);
    if (e == cudaSuccess && phase_ms) e = cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = launch_chain(p, w, kModeInvit, nullptr, 0, st);
    if (e == cudaSuccess && p.method == TINV_CWY) e = launch_finalize(p, w, st);
    if (e == cudaSuccess && phase_ms) e = cudaEventRecord(ev[4], st);
    if (e == cudaSuccess && phase_ms) {
        e = cudaEventSynchronize(ev[4]);
        for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&phase_ms[i], ev[i], ev[i + 1]);
    }
    for (int i = 0; i < 5; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    return cuda_code(e);
}

// Sizes and problem table of a batch (host arrays n, off_de, off_z), with the argument checks
// that need no array contents.  Returns 0 or the error code.
int batch_tables(int64_t nprob, const int64_t* n, const int64_t* off_de, const int64_t* off_z,
                 const uint64_t* seeds, const tinv_opts& o, int32_t P, Dims* D,
                 std::vector<Seg>* segs)
{
    Dims d;
    memset(&d, 0, sizeof(d));
    d.nseg = nprob;
    d.P = P;
    d.block = opts_block(o);
    segs->assign((size_t)nprob, Seg{});
    for (int64_t q = 0; q < nprob; ++q) {
        const int64_t nq = n[q];
        if (nq < 0 || nq > (int64_t)INT32_MAX / 2) return -2;
        if (off_de[q] < 0) return -3;
        if (off_z[q] < 0) return -4;
        Seg& g = (*segs)[(size_t)q];
        g.n = nq;
        g.m = nq;
        g.de = off_de[q];
        g.wo = off_de[q];
        g.z = off_z[q];
        g.ldz = nq > 0 ? nq : 1;
        g.j0 = d.M;
        g.foff = d.F;
        g.kj0 = o.j0;
        g.seed = seeds ? seeds[q] : o.seed;
        d.nmax = nq > d.nmax ? nq : d.nmax;
        d.M += nq;
        d.F += nq * nq;
        d.TT += nq * nq;
    }
    if (d.M > (int64_t)INT32_MAX / 2) return TINV_ENOTSUP;
    if (d.nmax < 1) d.nmax = 1;
    *D = d;
    return 0;
}

}  // namespace

namespace tinvx {

int batch_enqueue_device(int64_t nprob, const int64_t* n, const int64_t* off_de,
                         const int64_t* off_z, const uint64_t* seeds, const double* d,
                         const double* e, const double* w, double* Z, int64_t* info,
                         const tinv_opts& o)
{
    int64_t nmax = 1;
    for (int64_t q = 0; q < nprob; ++q) nmax = n[q] > nmax ? n[q] : nmax;
    const int32_t P = chain_grid(o.grid_ctas, nmax);
    Dims D;
    std::vector<Seg> segs;
    int rc = batch_tables(nprob, n, off_de, off_z, seeds, o, P, &D, &segs);
    if (rc != 0) return rc;
    if (D.M == 0) return 0;
    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = D.nmax;
    p.method = o.method;
    p.spin_limit = (uint32_t)o.spin_limit;
    p.seg_preset = 1;
    p.nseg = nprob;
    p.M = D.M;
    for (int64_t q = 0; q < nprob; ++q) p.zlen = std::max(p.zlen, off_z[q] + n[q] * n[q]);
    p.d = d;
    p.e = e;
    p.w = w;
    p.Z = Z;
    p.iters = o.iters;
    const Layout L = make_layout(D, true);
    cudaStream_t st = (cudaStream_t)o.stream;
    DevBuf own;
    void* ws = o.workspace;
    if (ws) {
        if (o.workspace_bytes < L.total) return TINV_EWORKSPACE;
    } else {
        cudaError_t ce = own.alloc(L.total, st, true);
        if (ce != cudaSuccess) return TINV_ENOMEM;
        ws = own.p;
    }
    const Ws wsb = bind_layout(ws, L, D);
    if (!(o.table_ready && o.workspace)) {
        cudaError_t ce = cudaMemcpyAsync(wsb.segs, segs.data(), segs.size() * sizeof(Seg),
                                         cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) return cuda_code(ce);
    }
    rc = enqueue_tinv(p, ws, D, o.max_team, st, o.phase_ms);
    if (rc != 0) return rc;
    if (info) {
        k_finish_batch<<<(unsigned)((nprob + 255) / 256), 256, 0, st>>>(wsb.ctr, wsb.sinfo, nprob, info);
        if (cudaGetLastError() != cudaSuccess) return TINV_ECUDA;
    }
    if (o.info) {
        k_finish<<<1, 1, 0, st>>>(wsb.ctr, o.info);
        if (cudaGetLastError() != cudaSuccess) return TINV_ECUDA;
    }
    if (o.counters) {
        k_counters<<<1, 1, 0, st>>>(wsb.ctr, o.counters);
        if (cudaGetLastError() != cudaSuccess) return TINV_ECUDA;
    }
    return 0;
}

size_t batch_workspace_bytes(int64_t nprob, const int64_t* n, const tinv_opts& o)
{
    int64_t nmax = 1;
    for (int64_t q = 0; q < nprob; ++q) nmax = n[q] > nmax ? n[q] : nmax;
    std::vector<int64_t> zeros((size_t)(nprob > 0 ? nprob : 1), 0);
    Dims D;
    std::vector<Seg> segs;
    if (batch_tables(nprob, n, zeros.data(), zeros.data(), nullptr, o, chain_grid(o.grid_ctas, nmax),
                     &D, &segs) != 0)
        return 0;
    return make_layout(D, true).total;
}

}  // namespace tinvx

extern "C" {

void tinv_opts_default(tinv_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->method = TINV_CWY;
}

const char* tinv_strerror(int code)
{
    switch (code) {
    case TINV_OK: return "success";
    case TINV_ENOMEM: return "device memory allocation failed";
    case TINV_ECUDA: return "CUDA runtime error";
    case TINV_ETIMEDOUT: return "a bounded device-side wait expired";
    case TINV_EINTERNAL: return "a device-side bounds check failed (debug build)";
    case TINV_EAGAIN: return "no capacity right now; retry";
    case TINV_ECANCELED: return "request cancelled";
    case TINV_ENOTSUP: return "size not supported by this library";
    case TINV_ENODEV: return "no usable sm_103 CUDA device";
    case TINV_EWORKSPACE: return "workspace too small";
    default: break;
    }
    if (code < 0) return "invalid argument";
    return "some eigenvectors did not converge";
}

const char* tinv_version(void) { return "tinv 0.2 (sm_103a, FP64)"; }

size_t tinv_workspace_size(int64_t n, int64_t m, const tinv_opts* o)
{
    if (n < 0 || m < 0) return 0;
    const Opts op(o);
    const int32_t P = chain_grid(op.o.grid_ctas, n);
    return make_layout(single_dims(n, m, P, opts_block(op.o)), true).total;
}

int tinv_ex(int64_t n, const double* d, const double* e, int64_t m, const double* w, double* Z,
            int64_t ldz, const tinv_opts* o, int64_t* ifail)
{
    const Opts op(o);
    if (n < 0) return -1;
    if (n > 0 && !d) return -2;
    if (n > 1 && !e) return -3;
    if (m < 0 || m > n) return -4;
    if (m > 0 && !w) return -5;
    if (m > 0 && !Z) return -6;
    if (ldz < (n > 0 ? n : 1)) return -7;
    if (op.o.method != TINV_CWY && op.o.method != TINV_MGS) return -8;
    if (n == 0 || m == 0) return 0;
    if (n > (int64_t)INT32_MAX / 2 || m > (int64_t)INT32_MAX / 2) return TINV_ENOTSUP;

    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.m = m;
    p.ldz = ldz;
    p.method = op.o.method;
    p.spin_limit = (uint32_t)op.o.spin_limit;
    p.seed = op.o.seed;
    p.j0 = op.o.j0;
    p.nseg = 1;
    p.M = m;
    const int32_t P = chain_grid(op.o.grid_ctas, n);
    const Dims D = single_dims(n, m, P, opts_block(op.o));

    if (op.o.device_ptrs) {
        cudaStream_t st = (cudaStream_t)op.o.stream;
        if (n == 1) {
            std::vector<double> ones(m, 0.0);
            for (int64_t j = 0; j < m; ++j) {
                const double one = 1.0;
                cudaError_t ce = cudaMemcpyAsync(Z + j * ldz, &one, sizeof(double),
                                                 cudaMemcpyHostToDevice, st);
                if (ce != cudaSuccess) return cuda_code(ce);
            }
            cudaStreamSynchronize(st);
            return 0;
        }
        p.d = d;
        p.e = e;
        p.w = w;
        p.Z = Z;
        p.iters = op.o.iters;
        const size_t need = make_layout(D, true).total;
        DevBuf own;
        void* ws = op.o.workspace;
        if (ws) {
            if (op.o.workspace_bytes < need) return TINV_EWORKSPACE;
        } else {
            cudaError_t ce = own.alloc(need, st, true);
            if (ce != cudaSuccess) return TINV_ENOMEM;
            ws = own.p;
        }
        int rc = enqueue_tinv(p, ws, D, op.o.max_team, st, op.o.phase_ms);
        if (rc != 0) return rc;
        const Ws wsb = bind_layout(ws, make_layout(D, true), D);
        if (op.o.info) {
            k_finish<<<1, 1, 0, st>>>(wsb.ctr, op.o.info);
            if (cudaGetLastError() != cudaSuccess) return TINV_ECUDA;
        }
        if (op.o.counters) {
            k_counters<<<1, 1, 0, st>>>(wsb.ctr, op.o.counters);
            if (cudaGetLastError() != cudaSuccess) return TINV_ECUDA;
        }
        return 0;
    }

    // ---- host pointers: validate values, copy in, run, copy out ----
    if (!all_finite(d, n) || (n > 1 && !all_finite(e, n - 1))) return -2;
    if (!all_finite(w, m)) return -5;
    if (!ascending(w, m)) return -5;
    if (n == 1) {
        for (int64_t j = 0; j < m; ++j) Z[j * ldz] = 1.0;
        return 0;
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
    int rc = 0;
    {
        const Layout L = make_layout(D, true);
        DevBuf dd, de, dw, dz, dit, ws;
        cudaError_t ce = dd.alloc(n * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = de.alloc((n - 1) * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dw.alloc(m * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dz.alloc((size_t)n * m * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dit.alloc(m * sizeof(int32_t), st, true);
        if (ce == cudaSuccess) ce = ws.alloc(L.total, st, true);
        if (ce != cudaSuccess) rc = TINV_ENOMEM;
        if (!rc) {
            ce = cudaMemcpyAsync(dd.p, d, n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(de.p, e, (n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(dw.p, w, m * sizeof(double), cudaMemcpyHostToDevice, st);
            rc = cuda_code(ce);
        }
        if (!rc) {
            p.d = (const double*)dd.p;
            p.e = (const double*)de.p;
            p.w = (const double*)dw.p;
            p.Z = (double*)dz.p;
            p.ldz = n;
            p.iters = (int32_t*)dit.p;
            rc = enqueue_tinv(p, ws.p, D, op.o.max_team, st, op.o.phase_ms);
        }
        int64_t ctr[kCtrCount];
        std::vector<int32_t> its(m);
        if (!rc) {
            const Ws wsb = bind_layout(ws.p, L, D);
            ce = cudaMemcpy2DAsync(Z, ldz * sizeof(double), dz.p, n * sizeof(double),
                                   n * sizeof(double), m, cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(ctr, wsb.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(its.data(), dit.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
        if (!rc) {
            if (op.o.counters) host_counters(ctr, op.o.counters);
            if (ctr[kCtrErr]) {
                rc = (int)err_code(ctr[kCtrErr]);
            } else {
                int64_t cnt = 0;
                for (int64_t j = 0; j < m; ++j) {
                    if (its[j] < 0) {
                        if (ifail) ifail[cnt] = j;
                        ++cnt;
                    }
                }
                if (op.o.iters)
                    for (int64_t j = 0; j < m; ++j) op.o.iters[j] = its[j];
                rc = (int)cnt;
            }
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}

int tinv(int64_t n, const double* d, const double* e, const double* w, double* Z)
{
    return tinv_ex(n, d, e, n, w, Z, n > 0 ? n : 1, nullptr, nullptr);
}

size_t tinv_batch_workspace_size(int64_t nprob, const int64_t* n, const tinv_opts* o)
{
    if (nprob < 0 || (nprob > 0 && !n)) return 0;
    const Opts op(o);
    int64_t nmax = 1;
    for (int64_t q = 0; q < nprob; ++q) nmax = n[q] > nmax ? n[q] : nmax;
    std::vector<int64_t> zeros((size_t)(nprob > 0 ? nprob : 1), 0);
    Dims D;
    std::vector<Seg> segs;
    if (batch_tables(nprob, n, zeros.data(), zeros.data(), nullptr, op.o,
                     chain_grid(op.o.grid_ctas, nmax), &D, &segs) != 0)
        return 0;
    return make_layout(D, true).total;
}

int tinv_batch(int64_t nprob, const int64_t* n, const int64_t* off_de, const int64_t* off_z,
               const double* d, const double* e, const double* w, double* Z, int64_t* info,
               const tinv_opts* o)
{
    const Opts op(o);
    if (nprob < 0) return -1;
    if (nprob == 0) return 0;
    if (!n) return -2;
    if (!off_de) return -3;
    if (!off_z) return -4;
    if (op.o.method != TINV_CWY && op.o.method != TINV_MGS) return -10;
    int64_t nmax = 1, de_len = 0, e_len = 0, z_len = 0;
    for (int64_t q = 0; q < nprob; ++q) {
        if (n[q] < 0) return -2;
        nmax = n[q] > nmax ? n[q] : nmax;
        if (n[q] == 0) continue;
        de_len = off_de[q] + n[q] > de_len ? off_de[q] + n[q] : de_len;
        e_len = off_de[q] + n[q] - 1 > e_len ? off_de[q] + n[q] - 1 : e_len;
        z_len = off_z[q] + n[q] * n[q] > z_len ? off_z[q] + n[q] * n[q] : z_len;
    }
    if (de_len > 0 && !d) return -5;
    if (e_len > 0 && !e) return -6;
    if (de_len > 0 && !w) return -7;
    if (z_len > 0 && !Z) return -8;
    if (op.o.device_ptrs)
        return batch_enqueue_device(nprob, n, off_de, off_z, nullptr, d, e, w, Z, info, op.o);
    const int32_t P = chain_grid(op.o.grid_ctas, nmax);
    Dims D;
    std::vector<Seg> segs;
    int rc = batch_tables(nprob, n, off_de, off_z, nullptr, op.o, P, &D, &segs);
    if (rc != 0) return rc;
    if (D.M == 0) return 0;

    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = D.nmax;
    p.method = op.o.method;
    p.spin_limit = (uint32_t)op.o.spin_limit;
    p.seg_preset = 1;
    p.nseg = nprob;
    p.M = D.M;
    for (int64_t q = 0; q < nprob; ++q) p.zlen = std::max(p.zlen, off_z[q] + n[q] * n[q]);
    const Layout L = make_layout(D, true);

    // ---- host pointers: validate values, copy in, run, copy out ----
    for (int64_t q = 0; q < nprob; ++q) {
        const int64_t nq = n[q];
        if (nq == 0) continue;
        if (!all_finite(d + off_de[q], nq)) return -5;
        if (nq > 1 && !all_finite(e + off_de[q], nq - 1)) return -6;
        if (!all_finite(w + off_de[q], nq) || !ascending(w + off_de[q], nq)) return -7;
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
    rc = 0;
    {
        DevBuf dd, de, dw, dz, dit, ws;
        cudaError_t ce = dd.alloc((size_t)de_len * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = de.alloc((size_t)(e_len > 0 ? e_len : 1) * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dw.alloc((size_t)de_len * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dz.alloc((size_t)z_len * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dit.alloc((size_t)D.M * sizeof(int32_t), st, true);
        if (ce == cudaSuccess) ce = ws.alloc(L.total, st, true);
        if (ce != cudaSuccess) rc = TINV_ENOMEM;
        const Ws wsb = bind_layout(ws.p, L, D);
        if (!rc) {
            ce = cudaMemcpyAsync(dd.p, d, (size_t)de_len * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && e_len > 0)
                ce = cudaMemcpyAsync(de.p, e, (size_t)e_len * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(dw.p, w, (size_t)de_len * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(wsb.segs, segs.data(), segs.size() * sizeof(Seg),
                                     cudaMemcpyHostToDevice, st);
            rc = cuda_code(ce);
        }
        if (!rc) {
            p.d = (const double*)dd.p;
            p.e = (const double*)de.p;
            p.w = (const double*)dw.p;
            p.Z = (double*)dz.p;
            p.iters = (int32_t*)dit.p;
            rc = enqueue_tinv(p, ws.p, D, op.o.max_team, st, op.o.phase_ms);
        }
        int64_t ctr[kCtrCount];
        std::vector<int64_t> sinfo((size_t)nprob);
        std::vector<int32_t> its;
        if (!rc) {
            for (int64_t q = 0; q < nprob && ce == cudaSuccess; ++q)
                if (n[q] > 0)
                    ce = cudaMemcpyAsync(Z + off_z[q], (double*)dz.p + off_z[q],
                                         (size_t)(n[q] * n[q]) * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(ctr, wsb.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(sinfo.data(), wsb.sinfo, (size_t)nprob * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess && op.o.iters)
                ce = cudaMemcpyAsync(op.o.iters, dit.p, (size_t)D.M * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
        if (!rc) {
            if (op.o.counters) host_counters(ctr, op.o.counters);
            if (ctr[kCtrErr]) {
                rc = (int)err_code(ctr[kCtrErr]);
                if (info)
                    for (int64_t q = 0; q < nprob; ++q) info[q] = rc;
            } else {
                int64_t cnt = 0;
                for (int64_t q = 0; q < nprob; ++q) {
                    if (info) info[q] = sinfo[(size_t)q];
                    cnt += sinfo[(size_t)q];
                }
                rc = cnt > INT32_MAX ? INT32_MAX : (int)cnt;
            }
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}

int tinv_plan(int64_t n, const double* d, const double* e, int64_t m, const double* w,
              double* wp, int32_t* head, double* scal, const tinv_opts* o)
{
    const Opts op(o);
    if (n < 1) return -1;
    if (!d) return -2;
    if (n > 1 && !e) return -3;
    if (m < 0 || m > n) return -4;
    if (m > 0 && !w) return -5;
    if (m > 0 && !wp) return -6;
    if (m > 0 && !head) return -7;
    if (!scal) return -8;
    const int32_t P = chain_grid(op.o.grid_ctas, n);
    const Dims D = single_dims(n, m, P);
    const Layout L = make_layout(D, false);
    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.m = m;
    p.ldz = n;
    p.method = op.o.method;
    p.nseg = 1;
    p.M = m;
    cudaStream_t st = op.o.device_ptrs ? (cudaStream_t)op.o.stream : nullptr;
    bool own_stream = false;
    if (!op.o.device_ptrs) {
        if (!all_finite(d, n) || (n > 1 && !all_finite(e, n - 1))) return -2;
        if (!all_finite(w, m) || !ascending(w, m)) return -5;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
        own_stream = true;
    }
    int rc = 0;
    {
        DevBuf ws, dd, de, dw;
        cudaError_t ce = ws.alloc(L.total, st, true);
        if (ce == cudaSuccess && !op.o.device_ptrs) {
            ce = dd.alloc(n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = de.alloc((n > 1 ? n - 1 : 1) * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = dw.alloc((m > 0 ? m : 1) * sizeof(double), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(dd.p, d, n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && n > 1)
                ce = cudaMemcpyAsync(de.p, e, (n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && m > 0)
                ce = cudaMemcpyAsync(dw.p, w, m * sizeof(double), cudaMemcpyHostToDevice, st);
            p.d = (const double*)dd.p;
            p.e = (const double*)de.p;
            p.w = (const double*)dw.p;
        } else {
            p.d = d;
            p.e = e;
            p.w = w;
        }
        rc = cuda_code(ce);
        const Ws wsb = bind_layout(ws.p, L, D);
        if (!rc) rc = cuda_code(launch_plan(p, wsb, 0, st));
        if (!rc) {
            const cudaMemcpyKind k = op.o.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            ce = cudaMemcpyAsync(scal, wsb.scal, 3 * sizeof(double), k, st);
            if (ce == cudaSuccess && m > 0) ce = cudaMemcpyAsync(wp, wsb.wp, m * sizeof(double), k, st);
            if (ce == cudaSuccess && m > 0)
                ce = cudaMemcpyAsync(head, wsb.head, m * sizeof(int32_t), k, st);
            if (ce == cudaSuccess && !op.o.device_ptrs) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
    }
    if (own_stream) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int tinv_lu(int64_t n, const double* d, const double* e, int64_t m, const double* s, double* l,
            double* u0, double* u1, double* u2, uint8_t* piv, const tinv_opts* o)
{
    const Opts op(o);
    if (n < 1) return -1;
    if (!d) return -2;
    if (n > 1 && !e) return -3;
    if (m < 0) return -4;
    if (m > 0 && !s) return -5;
    if (m > 0 && (!l || !u0 || !u1 || !u2 || !piv)) return -6;
    if (m == 0) return 0;
    if (op.o.device_ptrs) {
        cudaStream_t st = (cudaStream_t)op.o.stream;
        return cuda_code(launch_lu(n, d, e, m, s, l, u0, u1, u2, piv, nullptr, nullptr, st));
    }
    if (!all_finite(d, n) || (n > 1 && !all_finite(e, n - 1))) return -2;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
    int rc = 0;
    {
        const size_t mn = (size_t)m * (size_t)n;
        DevBuf dd, de, ds, dl, d0, d1, d2, dp;
        cudaError_t ce = dd.alloc(n * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = de.alloc((n > 1 ? n - 1 : 1) * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = ds.alloc(m * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dl.alloc(mn * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = d0.alloc(mn * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = d1.alloc(mn * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = d2.alloc(mn * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = dp.alloc(mn, st, true);
        if (ce != cudaSuccess) rc = TINV_ENOMEM;
        if (!rc) {
            ce = cudaMemcpyAsync(dd.p, d, n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && n > 1)
                ce = cudaMemcpyAsync(de.p, e, (n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(ds.p, s, m * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = launch_lu(n, (double*)dd.p, (double*)de.p, m, (double*)ds.p, (double*)dl.p,
                               (double*)d0.p, (double*)d1.p, (double*)d2.p, (uint8_t*)dp.p, nullptr,
                               nullptr, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(l, dl.p, mn * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(u0, d0.p, mn * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(u1, d1.p, mn * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(u2, d2.p, mn * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(piv, dp.p, mn, cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}

int tinv_solve(int64_t n, const double* d, const double* e, int64_t m, const double* s,
               double* X, int64_t ldx, int32_t scale, const tinv_opts* o)
{
    const Opts op(o);
    if (n < 1) return -1;
    if (!d) return -2;
    if (n > 1 && !e) return -3;
    if (m < 0) return -4;
    if (m > 0 && !s) return -5;
    if (m > 0 && !X) return -6;
    if (ldx < n) return -7;
    if (m == 0) return 0;
    const int32_t P = chain_grid(op.o.grid_ctas, n);
    const Dims D = single_dims(n, m, P);
    const Layout L = make_layout(D, false, true);
    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.m = m;
    cudaStream_t st = op.o.device_ptrs ? (cudaStream_t)op.o.stream : nullptr;
    bool own_stream = false;
    if (!op.o.device_ptrs) {
        if (!all_finite(d, n) || (n > 1 && !all_finite(e, n - 1))) return -2;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
        own_stream = true;
    }
    int rc = 0;
    {
        DevBuf ws, dd, de, ds, dx;
        cudaError_t ce = ws.alloc(L.total, st, true);
        double* X_dev = X;
        int64_t ldx_dev = ldx;
        if (ce == cudaSuccess && !op.o.device_ptrs) {
            ce = dd.alloc(n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = de.alloc((n > 1 ? n - 1 : 1) * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = ds.alloc(m * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = dx.alloc((size_t)n * m * sizeof(double), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(dd.p, d, n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess && n > 1)
                ce = cudaMemcpyAsync(de.p, e, (n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(ds.p, s, m * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpy2DAsync(dx.p, n * sizeof(double), X, ldx * sizeof(double),
                                       n * sizeof(double), m, cudaMemcpyHostToDevice, st);
            p.d = (const double*)dd.p;
            p.e = (const double*)de.p;
            X_dev = (double*)dx.p;
            ldx_dev = n;
            p.w = (const double*)ds.p;
        } else {
            p.d = d;
            p.e = e;
            p.w = s;
        }
        rc = cuda_code(ce);
        const Ws wsb = bind_layout(ws.p, L, D);
        if (!rc) rc = cuda_code(launch_norm(p, wsb, st));
        if (!rc)
            rc = cuda_code(launch_lu(n, p.d, p.e, m, p.w, wsb.fl, wsb.fr, wsb.fu1, wsb.fu2, wsb.fpiv,
                                     wsb.u0n, wsb.tolv, st));
        if (!rc) rc = cuda_code(launch_solve_rhs(n, m, wsb, X_dev, ldx_dev, scale, st));
        if (!rc && !op.o.device_ptrs) {
            ce = cudaMemcpy2DAsync(X, ldx * sizeof(double), X_dev, n * sizeof(double),
                                   n * sizeof(double), m, cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
    }
    if (own_stream) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

int tinv_orth(int64_t n, int64_t m, const double* V, int64_t ldv, double* Q, int64_t ldq,
              double* Y, double* T, const tinv_opts* o)
{
    const Opts op(o);
    if (n < 1) return -1;
    if (m < 0 || m > n) return -2;
    if (m > 0 && !V) return -3;
    if (ldv < n) return -4;
    if (m > 0 && !Q) return -5;
    if (ldq < n) return -6;
    if (op.o.method != TINV_CWY && op.o.method != TINV_MGS) return -9;
    if (m == 0) return 0;
    int32_t P = chain_grid(op.o.grid_ctas, n);
    const Dims D = single_dims(n, m, P, opts_block(op.o));
    const Layout L = make_layout(D, true);
    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.m = m;
    p.method = op.o.method;
    p.spin_limit = (uint32_t)op.o.spin_limit;
    p.nseg = 1;
    p.M = m;
    cudaStream_t st = op.o.device_ptrs ? (cudaStream_t)op.o.stream : nullptr;
    bool own_stream = false;
    if (!op.o.device_ptrs) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
        own_stream = true;
    }
    int rc = 0;
    {
        DevBuf ws, dv, dq;
        cudaError_t ce = ws.alloc(L.total, st, true);
        const double* V_dev = V;
        int64_t ldv_dev = ldv;
        if (ce == cudaSuccess && !op.o.device_ptrs) {
            ce = dv.alloc((size_t)n * m * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = dq.alloc((size_t)n * m * sizeof(double), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpy2DAsync(dv.p, n * sizeof(double), V, ldv * sizeof(double),
                                       n * sizeof(double), m, cudaMemcpyHostToDevice, st);
            V_dev = (const double*)dv.p;
            ldv_dev = n;
            p.Z = (double*)dq.p;
            p.ldz = n;
        } else {
            p.Z = Q;
            p.ldz = ldq;
        }
        p.zlen = (m - 1) * p.ldz + n;
        rc = cuda_code(ce);
        Ws wsb = bind_layout(ws.p, L, D);
        // team size for one cluster of m columns: at most n/16 CTAs and kTeamMax
        int32_t g = (int32_t)((n / 16 < (int64_t)P) ? (n / 16) : P);
        if (g > kTeamMax) g = kTeamMax;
        if (g >= 2 && op.o.method == TINV_CWY) {
            wsb.P = g;
        } else {
            wsb.P = 1;
        }
        if (op.o.max_team > 0 && wsb.P > op.o.max_team) wsb.P = op.o.max_team;
        if (wsb.P < 1) wsb.P = 1;
        if (!rc) rc = cuda_code(launch_orth_plan(p, wsb, p.method, st));
        if (!rc) rc = cuda_code(launch_chain(p, wsb, kModeOrth, V_dev, ldv_dev, st));
        const cudaMemcpyKind k = op.o.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (!rc && !op.o.device_ptrs) {
            ce = cudaMemcpy2DAsync(Q, ldq * sizeof(double), p.Z, n * sizeof(double),
                                   n * sizeof(double), m, cudaMemcpyDeviceToHost, st);
            rc = cuda_code(ce);
        }
        if (!rc && Y && op.o.method == TINV_CWY)
            rc = cuda_code(cudaMemcpyAsync(Y, wsb.Y, (size_t)n * m * sizeof(double), k, st));
        if (!rc && T && op.o.method == TINV_CWY)
            rc = cuda_code(cudaMemcpyAsync(T, wsb.T, (size_t)m * m * sizeof(double), k, st));
        if (!rc && !op.o.device_ptrs) {
            int64_t ctr[kCtrCount];
            ce = cudaMemcpyAsync(ctr, wsb.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
            if (!rc && ctr[kCtrErr]) rc = (int)err_code(ctr[kCtrErr]);
        }
    }
    if (own_stream) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    return rc;
}

}  // extern "C"
