// tinv_device.cuh -- device helpers of libtinv: start vectors, reductions, the bounded team
// barrier, the chunked tridiagonal solve, and the CTA-wide matrix-vector products used by the
// compact-WY and MGS reorthogonalization.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tinv_internal.h"

namespace tinvx {

constexpr double kEps = 2.220446049250313080847e-16;  // 2^-52, DBL_EPSILON
constexpr int kMaxIts = 5;   // DSTEIN MAXITS
constexpr int kExtra = 2;    // DSTEIN EXTRA: successes needed = EXTRA + 1
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kSpinTimeoutNs = 20ull * 1000 * 1000 * 1000;  // 20 s per barrier wait
constexpr uint32_t kSpinLimit = 400u * 1000 * 1000;            // and at most 4e8 polls

// ------------------------------------------------------------------------------------------
// Start vectors: SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based generator.
// Vector j, restart a: key = output (8j + a + 1) of the generator seeded with `seed`;
// element i = output (i + 1) of the generator seeded with `key`, mapped to [-1, 1).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t start_key(uint64_t seed, int64_t j, int attempt)
{
    return sm64_mix(seed + (uint64_t)(8 * j + attempt + 1) * kGamma);
}

__device__ __forceinline__ double start_value(uint64_t key, int64_t i)
{
    uint64_t x = sm64_mix(key + (uint64_t)(i + 1) * kGamma);
    double u01 = __dmul_rn(__ull2double_rn(x >> 11), 1.1102230246251565404e-16);  // * 2^-53
    return __dsub_rn(__dmul_rn(2.0, u01), 1.0);
}

__device__ __forceinline__ double sgn(double a) { return a < 0.0 ? -1.0 : 1.0; }

// ------------------------------------------------------------------------------------------
// Reductions (fixed shapes, so results do not depend on scheduling)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Largest |value| with the smallest index on ties; every lane receives the result.
__device__ __forceinline__ void warp_argmax(double& a, int64_t& idx)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double oa = __shfl_xor_sync(0xffffffffu, a, o);
        int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (oa > a || (oa == a && oi < idx)) {
            a = oa;
            idx = oi;
        }
    }
}

// CTA-wide sum / max; `sred` holds >= 33 doubles; every thread receives the result.
__device__ __forceinline__ double block_sum(double v, double* sred)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sred[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double s = lane < nw ? sred[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) sred[32] = s;
    }
    __syncthreads();
    return sred[32];
}

__device__ __forceinline__ double block_max(double v, double* sred)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sred[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double s = lane < nw ? sred[lane] : -1.0;
        s = warp_max(s);
        if (lane == 0) sred[32] = s;
    }
    __syncthreads();
    return sred[32];
}

// ------------------------------------------------------------------------------------------
// Bounded team barrier among G co-resident CTAs (a cooperative launch guarantees residency).
// `ctr` counts arrivals monotonically; the caller's `target` advances by G per barrier.  A
// wait gives up after kSpinTimeoutNs or kSpinLimit polls, sets the error word and returns
// false; callers unwind on false.  G == 1 is a plain CTA barrier.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p)
{
    return *(volatile const int*)p;
}

__device__ __noinline__ bool team_sync(uint32_t* ctr, uint32_t& target, int G, int* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (G <= 1) return ld_volatile_i32(err) == 0;
    if (threadIdx.x == 0) {
        target += (uint32_t)G;
        __threadfence();
        atomicAdd(ctr, 1u);
        int ok = 1;
        uint64_t t0 = globaltimer_ns();
        uint32_t spins = 0;
        while ((int32_t)(ld_acquire_u32(ctr) - target) < 0) {
            if (ld_volatile_i32(err) != 0) {
                ok = 0;
                break;
            }
            if (++spins > kSpinLimit || globaltimer_ns() - t0 > kSpinTimeoutNs) {
                atomicOr(err, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------------------------------
// Chunked solve of (T - s I) x = b with precomputed factors (in place on x).
//
// The P participating threads each own a contiguous chunk of L = ceil(n/P) rows.  Both
// substitutions are linear recurrences with fixed coefficients, so each chunk first computes
// its affine map (carry in -> carry out) in parallel, then one thread propagates the actual
// boundary values across the P chunks in order (values, not composed maps, so nothing grows
// beyond the true solution), then every chunk re-runs its rows from its true boundary value.
//
// Forward (P, L): carry c_k is the value at row k after the eliminations above it.
//   no interchange at k: y_k = c_k,      c_{k+1} = b_{k+1} - l_k c_k
//   interchange at k   : y_k = b_{k+1},  c_{k+1} = c_k - l_k b_{k+1}
// Back (U): x_k = (y_k - u1_k x_{k+1} - u2_k x_{k+2}) * r_k with r_k = 1/u0_k (perturbed).
//
// `sh` holds >= 8P doubles visible to the group; `t` is the thread's rank in the group (ranks
// >= P idle but must still call, because `sync` may be a CTA barrier).
// ------------------------------------------------------------------------------------------
struct Fac {
    const double* __restrict__ l;
    const double* __restrict__ u1;
    const double* __restrict__ u2;
    const double* __restrict__ r;
    const uint8_t* __restrict__ piv;
};

struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct CtaSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

template <class Sync>
__device__ void chunk_solve(int64_t n, const Fac& f, double* x, double* sh, int t, int P, Sync sync)
{
    const int64_t L = (n + P - 1) / P;
    const int64_t lo = (int64_t)t * L;
    const int64_t hi = (t < P) ? min(n, lo + L) : lo;
    const bool act = (t < P) && (lo < hi);
    double* mapA = sh;          // [P]  forward: multiplier of the incoming carry
    double* mapB = sh + P;      // [P]  forward: offset
    double* ent = sh + 6 * P;   // [2P] boundary values entering each chunk

    // ---- forward: phase 1, affine map of each chunk ----
    double A = 1.0, Bf = 0.0, bnext = 0.0;
    if (act) {
        for (int64_t k = lo; k < hi; ++k) {
            if (k + 1 < n) {
                const double b1 = x[k + 1];
                const double lk = f.l[k];
                if (f.piv[k]) {
                    Bf = fma(-lk, b1, Bf);
                } else {
                    A = -lk * A;
                    Bf = fma(-lk, Bf, b1);
                }
            }
        }
        if (hi < n) bnext = x[hi];
    }
    if (t < P) {
        mapA[t] = A;
        mapB[t] = Bf;
    }
    sync();
    // ---- forward: phase 2, boundary carries in order ----
    if (t == 0) {
        double c = x[0];
        for (int p = 0; p < P; ++p) {
            ent[p] = c;
            c = fma(mapA[p], c, mapB[p]);
        }
    }
    sync();
    // ---- forward: phase 3, rows of each chunk from the true carry ----
    if (act) {
        double c = ent[t];
        for (int64_t k = lo; k < hi; ++k) {
            if (k + 1 < n) {
                const double b1 = (k + 1 < hi) ? x[k + 1] : bnext;
                const double lk = f.l[k];
                if (f.piv[k]) {
                    x[k] = b1;
                    c = fma(-lk, b1, c);
                } else {
                    x[k] = c;
                    c = fma(-lk, c, b1);
                }
            } else {
                x[k] = c;
            }
        }
    }
    sync();

    // ---- back substitution: phase 1, particular + two homogeneous runs per chunk ----
    // state (cur, nxt) = (x_k, x_{k+1}) after processing row k; entering (x_hi, x_hi+1).
    double p0 = 0.0, p1 = 0.0, h10 = 1.0, h11 = 0.0, h20 = 0.0, h21 = 1.0;
    if (act) {
        for (int64_t k = hi - 1; k >= lo; --k) {
            const double rk = f.r[k], a = f.u1[k], b = f.u2[k], y = x[k];
            const double vp = fma(-b, p1, fma(-a, p0, y)) * rk;
            const double v1 = fma(-b, h11, -a * h10) * rk;
            const double v2 = fma(-b, h21, -a * h20) * rk;
            p1 = p0;
            p0 = vp;
            h11 = h10;
            h10 = v1;
            h21 = h20;
            h20 = v2;
        }
    }
    if (t < P) {
        sh[t] = h10;
        sh[P + t] = h20;
        sh[2 * P + t] = h11;
        sh[3 * P + t] = h21;
        sh[4 * P + t] = p0;
        sh[5 * P + t] = p1;
    }
    sync();
    // ---- back: phase 2, boundary values from the bottom chunk upwards ----
    if (t == 0) {
        double s0 = 0.0, s1 = 0.0;  // x_n = x_{n+1} = 0
        for (int p = P - 1; p >= 0; --p) {
            ent[2 * p] = s0;
            ent[2 * p + 1] = s1;
            const double n0 = fma(sh[p], s0, fma(sh[P + p], s1, sh[4 * P + p]));
            const double n1 = fma(sh[2 * P + p], s0, fma(sh[3 * P + p], s1, sh[5 * P + p]));
            s0 = n0;
            s1 = n1;
        }
    }
    sync();
    // ---- back: phase 3 ----
    if (act) {
        double cur = ent[2 * t], nxt = ent[2 * t + 1];
        for (int64_t k = hi - 1; k >= lo; --k) {
            const double v = fma(-f.u2[k], nxt, fma(-f.u1[k], cur, x[k])) * f.r[k];
            x[k] = v;
            nxt = cur;
            cur = v;
        }
    }
    sync();
}

// ------------------------------------------------------------------------------------------
// CTA-wide products used by the reorthogonalization.
//
// coldots: out(i, sum_{rho in R(i)} A[rho + i lda] x[rho]) for columns i in [c0, c1), with
//   R(i) = [max(rlo, i), rhi)    (LOWER: the nonzeros of a lower-trapezoidal column), or
//   R(i) = [rlo, min(rhi, i+1))  (UPPER: the nonzeros of an upper-triangular column).
// rowdots: out(rho, sum_{i in C(rho)} A[rho + i lda] x[i]) for rows rho in [r0, r1), with
//   C(rho) = [0, min(ccap, rho+1))  (LOWERCOL),  [rho, ccap)  (UPPERCOL),  [0, ccap)  (ALL).
// When there are fewer columns (rows) than threads, each is split into S segments whose
// partial sums are added in segment order; `red` holds >= 2*blockDim doubles.
// ------------------------------------------------------------------------------------------
enum ColKind { kLower = 0, kUpper = 1 };
enum RowKind { kLowerCol = 0, kUpperCol = 1, kAllCols = 2 };

template <int KIND, class Out>
__device__ void cta_coldots(const double* __restrict__ A, int64_t lda, int64_t c0, int64_t c1,
                            int64_t rlo, int64_t rhi, const double* x, double* red, Out out)
{
    const int B = blockDim.x, t = threadIdx.x;
    const int64_t nc = c1 - c0;
    if (nc <= 0) return;
    if (nc >= B) {
        for (int64_t i = c0 + t; i < c1; i += B) {
            const int64_t lo = (KIND == kLower) ? max(rlo, i) : rlo;
            const int64_t hi = (KIND == kLower) ? rhi : min(rhi, i + 1);
            const double* a = A + i * lda;
            double acc = 0.0;
            for (int64_t r = lo; r < hi; ++r) acc = fma(a[r], x[r], acc);
            out(i, acc);
        }
        __syncthreads();
        return;
    }
    int S = 1;
    while (S < 32 && (int64_t)(2 * S) * nc <= B) S *= 2;
    const int64_t ci = t % nc;
    const int sg = (int)(t / nc);
    if (sg < S) {
        const int64_t i = c0 + ci;
        const int64_t lo = (KIND == kLower) ? max(rlo, i) : rlo;
        const int64_t hi = (KIND == kLower) ? rhi : min(rhi, i + 1);
        const int64_t len = hi > lo ? hi - lo : 0;
        const int64_t seg = (len + S - 1) / S;
        const int64_t a0 = lo + sg * seg;
        const int64_t a1 = min(hi, a0 + seg);
        const double* a = A + i * lda;
        double acc = 0.0;
        for (int64_t r = a0; r < a1; ++r) acc = fma(a[r], x[r], acc);
        red[sg * nc + ci] = acc;
    }
    __syncthreads();
    if (t < nc) {
        double s = red[t];
        for (int q = 1; q < S; ++q) s += red[q * nc + t];
        out(c0 + t, s);
    }
    __syncthreads();
}

template <int KIND, int NV, class Out>
__device__ void cta_rowdots(const double* __restrict__ A, int64_t lda, int64_t r0, int64_t r1,
                            int64_t ccap, const double* x0, const double* x1, double* red, Out out)
{
    const int B = blockDim.x, t = threadIdx.x;
    const int64_t nr = r1 - r0;
    if (nr <= 0) return;
    if (nr >= B) {
        for (int64_t rho = r0 + t; rho < r1; rho += B) {
            const int64_t cb = (KIND == kUpperCol) ? rho : 0;
            const int64_t ce = (KIND == kLowerCol) ? min(ccap, rho + 1) : ccap;
            double acc0 = 0.0, acc1 = 0.0;
            for (int64_t i = cb; i < ce; ++i) {
                const double a = A[rho + i * lda];
                acc0 = fma(a, x0[i], acc0);
                if (NV == 2) acc1 = fma(a, x1[i], acc1);
            }
            out(rho, acc0, acc1);
        }
        __syncthreads();
        return;
    }
    int S = 1;
    while (S < 32 && (int64_t)(2 * S) * nr <= B) S *= 2;
    const int64_t ri = t % nr;
    const int sg = (int)(t / nr);
    if (sg < S) {
        const int64_t rho = r0 + ri;
        // fixed column grid over the columns any row of [r0, r1) can touch
        const int64_t gb = (KIND == kUpperCol) ? r0 : 0;
        const int64_t ge = (KIND == kLowerCol) ? min(ccap, r1) : ccap;
        const int64_t glen = ge > gb ? ge - gb : 0;
        const int64_t seg = (glen + S - 1) / S;
        const int64_t s0 = gb + sg * seg;
        const int64_t s1 = min(ge, s0 + seg);
        const int64_t cb = (KIND == kUpperCol) ? rho : 0;
        const int64_t ce = (KIND == kLowerCol) ? min(ccap, rho + 1) : ccap;
        double acc0 = 0.0, acc1 = 0.0;
        for (int64_t i = s0; i < s1; ++i) {
            if (i >= cb && i < ce) {
                const double a = A[rho + i * lda];
                acc0 = fma(a, x0[i], acc0);
                if (NV == 2) acc1 = fma(a, x1[i], acc1);
            }
        }
        red[(sg * nr + ri) * NV] = acc0;
        if (NV == 2) red[(sg * nr + ri) * NV + 1] = acc1;
    }
    __syncthreads();
    if (t < nr) {
        double s0 = red[t * NV], s1 = (NV == 2) ? red[t * NV + 1] : 0.0;
        for (int q = 1; q < S; ++q) {
            s0 += red[(q * nr + t) * NV];
            if (NV == 2) s1 += red[(q * nr + t) * NV + 1];
        }
        out(r0 + t, s0, s1);
    }
    __syncthreads();
}

}  // namespace tinvx
