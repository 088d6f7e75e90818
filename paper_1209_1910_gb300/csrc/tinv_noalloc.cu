// tinv_noalloc.cu -- tinv_solve_noalloc: the shifted tridiagonal solve (tinv_solve) for callers
// that must not have the library allocate device memory.
//
// Its scratch (the LU factors of every shift, the pivot bits and a few per-call scalars) lives
// in one file-scope __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.  Host code cannot pass that array's name to a kernel (on the host the
// name denotes a host-side stand-in, not device memory), so the device address is looked up once
// per device with cudaGetSymbolAddress, with that device current, and cached.
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

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up on the first call there).
cudaError_t noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
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
