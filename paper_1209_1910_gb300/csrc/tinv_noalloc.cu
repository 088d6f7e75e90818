// tinv_noalloc.cu -- tinv_solve_noalloc: the shifted tridiagonal solve (tinv_solve) for callers
// that must not have the library allocate device memory.
//
// Its scratch (the LU factors of every shift, the pivot bits and a few per-call scalars) lives
// in one file-scope __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.  Host code cannot pass that array's name to a kernel (on the host the
// name denotes a host-side stand-in, not device memory), so the device address is looked up with
// cudaGetSymbolAddress, with the device current, and cached.  A symbol's address belongs to a
// CUDA context (a driver context the caller made current, or a primary context re-created after
// cudaDeviceReset, has its own), so the cache is keyed by the unique id of the current context.
#include <cuda.h>
#include <mutex>
#include <string.h>

#include "../../include/tinv.h"
#include "tinv_internal.h"

using namespace tinvx;

namespace {

constexpr int64_t kNoAllocMaxElems = 262144;  // largest m * n accepted (e.g. 512 x 512)
constexpr int64_t kNoAllocMaxShifts = 131072; // largest m accepted
// 20 MiB holds the scratch layout of every (n, m) within both limits (largest: n = 2,
// m = 131072, about 16.8 MiB, of which the kept right-hand sides are 2 MiB)
constexpr size_t kNoAllocBytes = 20u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Context ids come from the driver API, reached through the runtime's entry-point lookup (the
// library does not link the driver library itself).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

constexpr int kCacheSize = 64;
struct CacheEntry {
    unsigned long long ctx_id;
    void* ptr;
};
std::mutex g_noalloc_mu;
CacheEntry g_noalloc_cache[kCacheSize] = {};
int g_noalloc_used = 0;
int g_noalloc_next = 0;  // slot replaced when the cache is full
bool g_noalloc_fn_init = false;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the current context; false when it cannot be determined.
bool current_context_id(unsigned long long* id)
{
    if (!g_noalloc_fn_init) {
        g_noalloc_fn_init = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = (CtxGetIdFn)f;
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch in the current context (looked up on the first call there).
cudaError_t noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    if (have_id) {
        for (int i = 0; i < g_noalloc_used; ++i)
            if (g_noalloc_cache[i].ctx_id == id) {
                *out = g_noalloc_cache[i].ptr;
                return cudaSuccess;
            }
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // also makes the primary context current
    if (e != cudaSuccess) return e;
    if (!have_id) have_id = current_context_id(&id);
    if (have_id) {
        int slot = g_noalloc_used < kCacheSize ? g_noalloc_used++ : (g_noalloc_next++ % kCacheSize);
        g_noalloc_cache[slot] = {id, p};
    }
    *out = p;
    return cudaSuccess;
}


}  // namespace

extern "C" int tinv_solve_noalloc(int64_t n, const double* d, const double* e, int64_t m,
                                  const double* s, double* X, int64_t ldx, int32_t scale,
                                  void* stream)
{
    if (n < 1) return -1;
    if (!d) return -2;
    if (n > 1 && !e) return -3;
    if (m < 0) return -4;
    if (m > 0 && !s) return -5;
    if (m > 0 && !X) return -6;
    if (ldx < n) return -7;
    if (m == 0) return 0;
    if (m > kNoAllocMaxShifts || m > kNoAllocMaxElems / n) return TINV_ENOTSUP;
    const int32_t P = 1;
    const Dims D = single_dims(n, m, P);
    const Layout L = make_layout(D, false, true);
    if (L.total > kNoAllocBytes) return TINV_ENOTSUP;
    void* base = nullptr;
    cudaError_t ce = noalloc_scratch(&base);
    if (ce != cudaSuccess) return cuda_code(ce);
    const Ws w = bind_layout(base, L, D);
    Problem p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.m = m;
    p.d = d;
    p.e = e;
    p.w = s;
    cudaStream_t st = (cudaStream_t)stream;
    // every scratch entry a call reads is written earlier in the same call (norm and counters
    // by the norm kernel, factors and thresholds by the LU kernels), so nothing is cleared
    ce = launch_norm(p, w, st);
    if (ce == cudaSuccess)
        ce = launch_lu(n, d, e, m, s, w.fl, w.fr, w.fu1, w.fu2, w.fpiv, w.u0n, w.tolv, st);
    if (ce == cudaSuccess) ce = launch_solve_rhs(n, m, w, X, ldx, scale, st);
    return cuda_code(ce);
}
