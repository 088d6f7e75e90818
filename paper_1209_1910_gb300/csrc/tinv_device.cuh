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

// Bounds check of TINV_DEBUG builds (see TINV_IN): false, with kErrBounds set, on failure.
__device__ __forceinline__ bool dbg_ok(bool cond, int* err)
{
    if (!cond) atomicOr(err, kErrBounds);
    return cond;
}
__device__ __forceinline__ bool dbg_range(int64_t lo, int64_t hi, int64_t cap)
{
    return 0 <= lo && lo <= hi && hi <= cap;
}

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
// wait gives up after kSpinTimeoutNs or `limit` polls (0 = kSpinLimit), sets the error word and
// returns false; callers unwind on false.  G == 1 is a plain CTA barrier.
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

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p)
{
    return *(volatile const unsigned long long*)p;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t* p, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __noinline__ bool team_sync(uint32_t* ctr, uint32_t& target, int G, int* err,
                                       uint32_t limit = 0)
{
    __shared__ int s_ok;
    __syncthreads();
    if (G <= 1) return ld_volatile_i32(err) == 0;
    if (threadIdx.x == 0) {
        target += (uint32_t)G;
        red_release_add_u32(ctr, 1u);  // the CTA's writes (ordered by the barrier) go first
        int ok = 1;
        uint64_t t0 = 0;
        uint32_t spins = 0;
        const uint32_t lim = limit ? limit : kSpinLimit;
        while ((int32_t)(ld_acquire_u32(ctr) - target) < 0) {
            ++spins;
            if ((spins & 63u) == 0 || spins >= lim) {
                if (ld_volatile_i32(err) != 0) {
                    ok = 0;
                    break;
                }
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                if (spins >= lim || now - t0 > kSpinTimeoutNs) {
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
            }
        }
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
// its affine map (carry in -> carry out) in parallel, then one thread propagates the boundary
// values across the P chunks in order, then every chunk re-runs its rows from its boundary
// value.  The forward maps compose the multipliers l (scaled pivoting lets |l| exceed 1; on the
// workloads measured their folds stay accurate, and they are not checked).  The
// back-substitution maps grow by
// 1/|u0| at every small pivot, and near-singular shifts of clustered spectra can put several
// small pivots into one chunk; the boundary value folded from such a map then carries an error
// far above the rounding of the true solution.  Every chunk therefore re-checks the rows next to
// its lower boundary against the values its neighbour computed (row_consistent); if any row
// fails, the solve is redone sequentially, so the result is always backward stable.
//
// Forward (P, L): carry c_k is the value at row k after the eliminations above it.
//   no interchange at k: y_k = c_k,      c_{k+1} = b_{k+1} - l_k c_k
//   interchange at k   : y_k = b_{k+1},  c_{k+1} = c_k - l_k b_{k+1}
// Back (U): x_k = a_k x_{k+1} + b_k x_{k+2} + r_k y_k with r_k = 1/u0_k (perturbed),
//   a_k = -u1_k r_k and b_k = -u2_k r_k (the factors are stored in this form).
//
// `sh` holds >= 8P doubles visible to the group; `t` is the thread's rank in the group (ranks
// >= P idle but must still call, because `sync` may be a CTA barrier).
// ------------------------------------------------------------------------------------------
struct Fac {
    const double* __restrict__ l;    // multipliers of L
    const double* __restrict__ a;    // -u1 / u0 (perturbed u0)
    const double* __restrict__ b;    // -u2 / u0
    const double* __restrict__ r;    // 1 / u0
    const uint8_t* __restrict__ piv; // row interchanges
};

// One row of the back substitution: x_k from x_{k+1}, x_{k+2} and the forward result y_k.
__device__ __forceinline__ double back_row(double a, double b, double r, double y, double x1, double x2)
{
    return fma(a, x1, fma(b, x2, y * r));
}

struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct CtaSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Sequential back substitution by the calling thread alone of rows [0, top), from the forward
// results y and the already final x[top], x[top + 1] (rows at or past n count as 0).  The
// parallel solves fall back to it when their consistency check fails, from the lowest failing
// chunk boundary: the rows below it passed every check, so they are already backward stable.
__device__ __noinline__ void seq_back(int64_t n, const Fac& f, const double* y, double* x, int64_t top)
{
    double cur = top < n ? x[top] : 0.0, nxt = top + 1 < n ? x[top + 1] : 0.0;
    int64_t k = top - 1;
    for (; k >= 3; k -= 4) {
        double a[4], b[4], z[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a[i] = f.a[k - i];
            b[i] = f.b[k - i];
            z[i] = y[k - i] * f.r[k - i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double v = fma(a[i], cur, fma(b[i], nxt, z[i]));
            x[k - i] = v;
            nxt = cur;
            cur = v;
        }
    }
    for (; k >= 0; --k) {
        const double v = back_row(f.a[k], f.b[k], f.r[k], y[k], cur, nxt);
        x[k] = v;
        nxt = cur;
        cur = v;
    }
}

// The same by a whole CTA: warps 1.. stream the coefficients (a, b, r y) of the next block of
// rows into shared memory while two lanes of warp 0 run the current block's recurrence from
// shared memory.  Row k is x_k = fma(a_k, x_{k+1}, t_k) with t_k = fma(b_k, x_{k+2}, r_k y_k);
// t_k needs only x_{k+2}, so lane 1 forms it while lane 0 forms x_{k+1}: one FP64 instruction
// for both lanes and one lane exchange per row (a single thread would issue two dependent FP64
// instructions per row).  The operations and their operands are those of seq_back, so the
// results are identical.  `sh` holds >= 6 kStageRows doubles.  Called by every thread of the
// CTA; y and x may be global or shared (not the same array).
constexpr int kStageRows = 320;
__device__ __noinline__ void staged_seq_back(int64_t n, const Fac& f, const double* y, double* x,
                                             double* sh, int64_t top0)
{
    const int t = threadIdx.x, B = blockDim.x;
    auto stage = [&](int64_t lo, int64_t hi, int buf, int t0, int nt) {
        double* sa = sh + buf * 3 * kStageRows;
        for (int64_t k = lo + (t - t0); k < hi; k += nt) {
            const int64_t i = k - lo;
            sa[i] = f.a[k];
            sa[kStageRows + i] = f.b[k];
            sa[2 * kStageRows + i] = y[k] * f.r[k];
        }
    };
    int64_t top = top0;
    int64_t lo = top > kStageRows ? top - kStageRows : 0;
    stage(lo, top, 0, 0, B);
    // lane 0: cur = x_{k+1}, nxt = x_{k+2}; lane 1: tk = t_k for the next row k
    double cur = 0.0, nxt = 0.0, tk = 0.0;
    if (t < 2) {
        cur = top < n ? x[top] : 0.0;
        nxt = top + 1 < n ? x[top + 1] : 0.0;
    }
    __syncthreads();
    for (int blk = 0;; ++blk) {
        const int64_t nlo = lo > kStageRows ? lo - kStageRows : 0;
        if (t >= 32 && lo > 0) stage(nlo, lo, (blk + 1) & 1, 32, B - 32);
        if (t < 2 && top > lo) {
            const double* sa = sh + (blk & 1) * 3 * kStageRows;
            const double* sb = sa + kStageRows;
            const double* sz = sa + 2 * kStageRows;
            // t for the block's first row from the values both lanes hold
            tk = fma(sb[top - 1 - lo], nxt, sz[top - 1 - lo]);
            for (int64_t k = top - 1; k >= lo; --k) {
                const int64_t i = k - lo;
                // lane 0 receives t_k, lane 1 receives x_{k+1}
                const double other = __shfl_xor_sync(0x3u, t == 0 ? cur : tk, 1);
                const double xk1 = (t == 0) ? cur : other;
                // lane 0: x_k = a_k x_{k+1} + t_k;  lane 1: t_{k-1} = b_{k-1} x_{k+1} + z_{k-1}
                // (row k-1 is in this block unless k == lo; that t is formed after the block)
                const int64_t j = (t == 0 || k == lo) ? i : i - 1;
                const double p = (t == 0) ? sa[j] : sb[j];
                const double c = (t == 0) ? other : sz[j];
                const double v = fma(p, xk1, c);
                if (t == 0) {
                    x[k] = v;
                    nxt = cur;
                    cur = v;
                } else {
                    tk = v;
                    nxt = xk1;  // x_{k+1}: after the block's last row, the next block's first t
                }
            }
        }
        __syncthreads();
        if (lo == 0) break;
        top = lo;
        lo = nlo;
    }
}

// Backward-stability test of one row of the back substitution: x_k recomputed from the stored
// neighbours x_{k+1}, x_{k+2} (and the row's right-hand side y) agrees with the stored x_k to a
// few roundings of the row's terms.  Rows inside a chunk pass by construction; a row next to a
// chunk boundary fails when the boundary values its chunk assumed (from the folded chunk maps,
// which lose accuracy when the maps grow across several tiny pivots) are not the values the
// neighbouring chunk computed.  A NaN or infinity fails.
#ifndef TINV_SOLVE_TOL
#define TINV_SOLVE_TOL 1024.0
#endif
constexpr double kSolveTol = TINV_SOLVE_TOL;  // accepted backward error of a row, in eps
// For a solve whose result only starts the next sweep (not a possible final vector) any error
// that leaves a usable start vector is harmless; this bound still rejects garbage.
constexpr double kSolveTolLoose = 1099511627776.0;  // 2^40 eps

__device__ __forceinline__ bool row_consistent(double a, double b, double r, double y, double x1,
                                               double x2, double xk, double tol)
{
    const double v = back_row(a, b, r, y, x1, x2);
    const double scale = fabs(y * r) + fabs(a * x1) + fabs(b * x2);
    return fabs(v - xk) <= tol * kEps * scale;
}

// x (n rows) solved in place by P chunks; `ysave` (n doubles) receives the forward results for
// the sequential fallback; `tol` is the accepted backward error of a row, in eps.  Returns true
// when the fallback ran.
template <class Sync>
__device__ bool chunk_solve(int64_t n, const Fac& f, double* x, double* ysave, double* sh, int t,
                            int P, Sync sync, double tol = kSolveTol)
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
            const double a = f.a[k], b = f.b[k], y = x[k];
            const double vp = back_row(a, b, f.r[k], y, p0, p1);
            const double v1 = fma(a, h10, b * h11);
            const double v2 = fma(a, h20, b * h21);
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
    double ysv0 = 0.0, ysv1 = 0.0;  // forward results of rows hi-1, hi-2
    if (act) {
        double cur = ent[2 * t], nxt = ent[2 * t + 1];
        ysv0 = x[hi - 1];
        if (hi - 2 >= lo) ysv1 = x[hi - 2];
        for (int64_t k = hi - 1; k >= lo; --k) {
            const double y = x[k];
            ysave[k] = y;
            const double v = back_row(f.a[k], f.b[k], f.r[k], y, cur, nxt);
            x[k] = v;
            nxt = cur;
            cur = v;
        }
    }
    sync();
    // ---- rows next to the chunk boundaries against the neighbours' values ----
    bool bad = false;
    if (act && hi < n) {
        const double x1 = x[hi], x2 = (hi + 1 < n) ? x[hi + 1] : 0.0;
        bad = !row_consistent(f.a[hi - 1], f.b[hi - 1], f.r[hi - 1], ysv0, x1, x2, x[hi - 1], tol);
        if (hi - 2 >= lo)
            bad = bad || !row_consistent(f.a[hi - 2], f.b[hi - 2], f.r[hi - 2], ysv1, x[hi - 1], x1,
                                         x[hi - 2], tol);
    }
    const bool fallback = __any_sync(0xffffffffu, bad);
    if (fallback) {
        // restart below the lowest failing boundary (the largest failing hi)
        const int top = __reduce_max_sync(0xffffffffu, bad ? (int)hi : 0);
        if (t == 0) seq_back(n, f, ysave, x, top);
        sync();
    }
    return fallback;
}

// ------------------------------------------------------------------------------------------
// Repair of a CTA's chunked back substitution (all rows of the system in x, the forward results
// in y) whose consistency check failed.  The rows at and below `top` passed; the chunk [top - L,
// top) that failed is redone sequentially from x[top], x[top + 1]; the rows above it are redone
// by a fresh chunked pass (128 chunks, one thread folding the chunk maps as values) from those
// values, and its chunk boundaries are checked again.  Returns 0 once every row passed, else,
// after kRepairRounds rounds, the row from which the sequential fallback must restart.  Called
// by every thread of the CTA; `sh` holds >= 1024 doubles.
// ------------------------------------------------------------------------------------------
constexpr int kRepairRounds = 4;
__device__ __noinline__ int64_t cta_back_repair(int64_t n, const Fac& f, const double* y, double* x,
                                                double* sh, int64_t top, int64_t L, double tol)
{
    constexpr int P = 128;
    const int t = threadIdx.x;
    __shared__ unsigned long long s_rtop;
    for (int round = 0; round < kRepairRounds; ++round) {
        const int64_t lo_f = max((int64_t)0, top - L);
        if (t == 0) {  // the failing chunk, sequentially
            double cur = top < n ? x[top] : 0.0, nxt = top + 1 < n ? x[top + 1] : 0.0;
            for (int64_t k = top - 1; k >= lo_f; --k) {
                const double v = back_row(f.a[k], f.b[k], f.r[k], y[k], cur, nxt);
                x[k] = v;
                nxt = cur;
                cur = v;
            }
        }
        __syncthreads();
        const int64_t R = lo_f;  // rows [0, R) remain, entering values x[R], x[R + 1]
        if (R <= 0) return 0;
        const int Pn = (int)min((int64_t)P, max((int64_t)1, R / 2));
        const int64_t Lc = (R + Pn - 1) / Pn;
        const int64_t clo = (int64_t)t * Lc;
        const int64_t chi = (t < Pn) ? min(R, clo + Lc) : clo;
        const bool act = (t < Pn) && (clo < chi);
        double p0 = 0.0, p1 = 0.0, h10 = 1.0, h11 = 0.0, h20 = 0.0, h21 = 1.0;
        if (act) {
            for (int64_t k = chi - 1; k >= clo; --k) {
                const double a = f.a[k], b = f.b[k];
                const double vp = back_row(a, b, f.r[k], y[k], p0, p1);
                const double v1 = fma(a, h10, b * h11);
                const double v2 = fma(a, h20, b * h21);
                p1 = p0;
                p0 = vp;
                h11 = h10;
                h10 = v1;
                h21 = h20;
                h20 = v2;
            }
        }
        if (t < Pn) {
            sh[t] = h10;
            sh[P + t] = h20;
            sh[2 * P + t] = h11;
            sh[3 * P + t] = h21;
            sh[4 * P + t] = p0;
            sh[5 * P + t] = p1;
        }
        __syncthreads();
        double* ent = sh + 6 * P;  // [2P] values entering each chunk
        if (t == 0) {
            double s0 = x[R], s1 = (R + 1 < n) ? x[R + 1] : 0.0;
            for (int q = Pn - 1; q >= 0; --q) {
                ent[2 * q] = s0;
                ent[2 * q + 1] = s1;
                const double n0 = fma(sh[q], s0, fma(sh[P + q], s1, sh[4 * P + q]));
                const double n1 = fma(sh[2 * P + q], s0, fma(sh[3 * P + q], s1, sh[5 * P + q]));
                s0 = n0;
                s1 = n1;
            }
        }
        __syncthreads();
        if (act) {
            double cur = ent[2 * t], nxt = ent[2 * t + 1];
            for (int64_t k = chi - 1; k >= clo; --k) {
                const double v = back_row(f.a[k], f.b[k], f.r[k], y[k], cur, nxt);
                x[k] = v;
                nxt = cur;
                cur = v;
            }
        }
        if (t == 0) s_rtop = 0ull;
        __syncthreads();
        // the boundaries between the new chunks (the top chunk started from exact values)
        bool bad = false;
        if (act && chi < R) {
            const double x1 = x[chi], x2 = x[chi + 1];
            bad = !row_consistent(f.a[chi - 1], f.b[chi - 1], f.r[chi - 1], y[chi - 1], x1, x2, x[chi - 1], tol);
            if (chi - 2 >= clo)
                bad = bad || !row_consistent(f.a[chi - 2], f.b[chi - 2], f.r[chi - 2], y[chi - 2], x[chi - 1], x1,
                                             x[chi - 2], tol);
        }
        if (bad) atomicMax(&s_rtop, (unsigned long long)chi);
        __syncthreads();
        top = (int64_t)s_rtop;
        __syncthreads();
        if (top == 0) return 0;
        L = Lc;
    }
    return top;
}

// ------------------------------------------------------------------------------------------
// Team-distributed solve of (T - s I) x = fac * b.
//
// The team's G CTAs each own rows [r0, r1) (>= 2 rows each).  Inside a CTA the first 128
// threads own contiguous chunks; every chunk computes the affine map of both substitutions
// over its rows (as in chunk_solve).  Maps are combined by an inclusive Kogge-Stone scan inside
// each warp, then by one thread over the 4 warps into the CTA's map, which is published to the
// team.  After one team barrier per direction every CTA folds the published maps of the CTAs
// before it (forward) or after it (back) as actual values.  In the forward direction the warps'
// composed maps then give every chunk its carry; in the back direction (whose maps grow at small
// pivots) the first lane of each warp folds the warp's own chunk maps as values instead.  Every
// chunk then re-runs its rows from its boundary values, and the result is checked.
//   bsrc  : right-hand side (global, or shared when G == 1); the solve reads bsrc[k] * fac for
//           its rows and the first row of the next CTA.
//   ysave : n doubles (global when G > 1, not vsm) receiving the forward results of the own rows,
//           which the sequential fallback reads for all rows.
//   vsm   : row-indexed scratch of the CTA (n slots); on return vsm[r0..r1) = x.
//   vout  : if not null, also receives x[r0..r1) (global, for other CTAs of the team).
//   pubf, pubb : team buffers of 2 and 6 doubles per rank for the published maps.
//   sh    : 2048 doubles of shared scratch (128 + 6 G + 6 * 128 are used; G <= 192).
// ------------------------------------------------------------------------------------------
struct TeamRef {
    uint32_t* bar;
    uint32_t* target;
    int G, rank;
    int* err;
    unsigned long long* flag;  // team word for the consistency verdict (G > 1)
    unsigned long long stamp;  // increasing per solve of the team
    unsigned long long* nfall; // counter of sequential fallbacks (may be null)
    double tol;                // accepted backward error of a row, in eps
    uint32_t limit;            // polls of a barrier wait (0 = default)
};

__device__ __forceinline__ void compose2(double& m00, double& m01, double& m10, double& m11,
                                         double& f0, double& f1, double n00, double n01,
                                         double n10, double n11, double g0, double g1)
{
    // (M, f) <- (M, f) o (N, g) = (M N, M g + f): apply (N, g) first
    const double a00 = fma(m00, n00, m01 * n10), a01 = fma(m00, n01, m01 * n11);
    const double a10 = fma(m10, n00, m11 * n10), a11 = fma(m10, n01, m11 * n11);
    const double b0 = fma(m00, g0, fma(m01, g1, f0)), b1 = fma(m10, g0, fma(m11, g1, f1));
    m00 = a00;
    m01 = a01;
    m10 = a10;
    m11 = a11;
    f0 = b0;
    f1 = b1;
}

// Scratch layout of the team solve with NW chunk warps (doubles of sh): forward warp maps,
// warp carries, back warp maps, warp entering values, the team's published maps (6 per rank),
// then the chunk maps (6 per chunk).
template <int NW>
struct SolveScratch {
    static constexpr int kFwd = 0, kCarry = 2 * NW, kWarp = 3 * NW, kEnter = 9 * NW;
    static constexpr int kPub = (11 * NW + 15) / 16 * 16;
    __device__ static constexpr int chunk_maps(int G) { return kPub + 6 * G; }
    __device__ static constexpr int size(int G) { return kPub + 6 * G + 6 * 32 * NW; }
};

#ifdef TINV_PHASE_PROFILE
// Diagnostic build: SM cycles of the 16-warp solve's steps, per CTA (thread 0's timeline).
constexpr int kSolvePh = 8;
__device__ unsigned long long g_solve_prof[1024 * kSolvePh];
#define SOLVE_MARK(i)                                                                    \
    do {                                                                                 \
        if (NW == 16 && threadIdx.x == 0) {                                              \
            const long long _n = clock64();                                              \
            g_solve_prof[blockIdx.x * kSolvePh + (i)] += (unsigned long long)(_n - _sp); \
            _sp = _n;                                                                    \
        }                                                                                \
    } while (0)
#else
#define SOLVE_MARK(i) \
    do {              \
    } while (0)
#endif

template <int NW>
__device__ __noinline__ bool team_solve_nw(int64_t n, const Fac& f, const double* bsrc, double fac,
                                           double* vsm, double* vout, double* ysave, int64_t r0,
                                           int64_t r1, double* pubf, double* pubb, TeamRef tr,
                                           double* sh)
{
    constexpr int PT = 32 * NW;
    using SS = SolveScratch<NW>;
    const int t = threadIdx.x, B = blockDim.x, lane = t & 31, wid = t >> 5;
    if (!TINV_IN(dbg_range(r0, r1, n) && r1 > r0 && tr.rank < tr.G && tr.G <= kTeamMax, tr.err))
        return false;
    const int64_t R = r1 - r0;
    const int Pn = (int)min((int64_t)PT, max((int64_t)1, R / 2));
    const int64_t L = (R + Pn - 1) / Pn;
    const bool part = t < PT;
    const int64_t lo = r0 + (int64_t)t * L;
    const int64_t hi = (t < Pn) ? min(r1, lo + L) : lo;
    const bool act = (t < Pn) && (lo < hi);
#ifdef TINV_PHASE_PROFILE
    long long _sp = clock64();
#endif

    // stage b (scaled) for the own rows and the first row of the next CTA
    const int64_t send = min(r1 + 1, n);
    for (int64_t k = r0 + t; k < send; k += B) vsm[k] = bsrc[k] * fac;
    __syncthreads();
    SOLVE_MARK(0);

    // ---------------- forward (P, L) ----------------
    double A = 1.0, Bf = 0.0, bnext = 0.0;
    if (act) {
        for (int64_t k = lo; k < hi; ++k) {
            if (k + 1 < n) {
                const double b1 = vsm[k + 1];
                const double lk = f.l[k];
                if (f.piv[k]) {
                    Bf = fma(-lk, b1, Bf);
                } else {
                    A = -lk * A;
                    Bf = fma(-lk, Bf, b1);
                }
            }
        }
        if (hi < n) bnext = vsm[hi];
    }
    double ea = 1.0, eb = 0.0;  // exclusive prefix map within the warp
    if (part) {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double pa = __shfl_up_sync(0xffffffffu, A, d);
            const double pb = __shfl_up_sync(0xffffffffu, Bf, d);
            if (lane >= d) {
                Bf = fma(A, pb, Bf);
                A = A * pa;
            }
        }
        ea = __shfl_up_sync(0xffffffffu, A, 1);
        eb = __shfl_up_sync(0xffffffffu, Bf, 1);
        if (lane == 0) {
            ea = 1.0;
            eb = 0.0;
        }
        if (lane == 31) {
            sh[SS::kFwd + 2 * wid] = A;
            sh[SS::kFwd + 2 * wid + 1] = Bf;
        }
    }
    __syncthreads();
    SOLVE_MARK(1);
    if (t == 0 && tr.G > 1) {
        double CA = 1.0, CB = 0.0;
        for (int w2 = 0; w2 < NW; ++w2) {
            CB = fma(sh[SS::kFwd + 2 * w2], CB, sh[SS::kFwd + 2 * w2 + 1]);
            CA = sh[SS::kFwd + 2 * w2] * CA;
        }
        pubf[2 * tr.rank] = CA;
        pubf[2 * tr.rank + 1] = CB;
    }
    if (!team_sync(tr.bar, *tr.target, tr.G, tr.err, tr.limit)) return false;
    double* pf = sh + SS::kPub;  // the published forward maps of the CTAs before this one
    for (int q = t; q < tr.rank; q += B) {
        pf[2 * q] = __ldcg(&pubf[2 * q]);
        pf[2 * q + 1] = __ldcg(&pubf[2 * q + 1]);
    }
    __syncthreads();
    if (t == 0) {
        double c;
        if (tr.rank == 0) {
            c = vsm[r0];
        } else {
            c = bsrc[0] * fac;
            for (int q = 0; q < tr.rank; ++q) c = fma(pf[2 * q], c, pf[2 * q + 1]);
        }
        for (int w2 = 0; w2 < NW; ++w2) {
            sh[SS::kCarry + w2] = c;
            c = fma(sh[SS::kFwd + 2 * w2], c, sh[SS::kFwd + 2 * w2 + 1]);
        }
    }
    __syncthreads();
    SOLVE_MARK(2);
    if (act) {
        double c = fma(ea, sh[SS::kCarry + wid], eb);
        for (int64_t k = lo; k < hi; ++k) {
            if (k + 1 < n) {
                const double b1 = (k + 1 < hi) ? vsm[k + 1] : bnext;
                const double lk = f.l[k];
                if (f.piv[k]) {
                    vsm[k] = b1;
                    c = fma(-lk, b1, c);
                } else {
                    vsm[k] = c;
                    c = fma(-lk, c, b1);
                }
            } else {
                vsm[k] = c;
            }
        }
    }
    __syncthreads();
    SOLVE_MARK(3);

    // ---------------- back substitution (U) ----------------
    // chunk map: (x_lo, x_lo+1) = M (x_hi, x_hi+1) + f
    double m00 = 1.0, m01 = 0.0, m10 = 0.0, m11 = 1.0, f0 = 0.0, f1 = 0.0;
    if (act) {
        double p0 = 0.0, p1 = 0.0, h10 = 1.0, h11 = 0.0, h20 = 0.0, h21 = 1.0;
        for (int64_t k = hi - 1; k >= lo; --k) {
            const double a = f.a[k], b = f.b[k], y = vsm[k];
            const double vp = back_row(a, b, f.r[k], y, p0, p1);
            const double v1 = fma(a, h10, b * h11);
            const double v2 = fma(a, h20, b * h21);
            p1 = p0;
            p0 = vp;
            h11 = h10;
            h10 = v1;
            h21 = h20;
            h20 = v2;
        }
        m00 = h10;
        m01 = h20;
        m10 = h11;
        m11 = h21;
        f0 = p0;
        f1 = p1;
    }
    // The chunks' own maps, kept for the value fold below that gives every chunk its boundary
    // values (applying composed maps to values loses accuracy when they span several small
    // pivots; the compositions are used only between warps and between CTAs).
    double* cm = sh + SS::chunk_maps(tr.G);  // [6 * PT]
    if (part) {
        double* o = cm + 6 * t;
        o[0] = m00;
        o[1] = m01;
        o[2] = m10;
        o[3] = m11;
        o[4] = f0;
        o[5] = f1;
    }
    // inclusive suffix scan within the warp: S_p = m_p o m_{p+1} o ... o m_31
    if (part) {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double n00 = __shfl_down_sync(0xffffffffu, m00, d);
            const double n01 = __shfl_down_sync(0xffffffffu, m01, d);
            const double n10 = __shfl_down_sync(0xffffffffu, m10, d);
            const double n11 = __shfl_down_sync(0xffffffffu, m11, d);
            const double q0 = __shfl_down_sync(0xffffffffu, f0, d);
            const double q1 = __shfl_down_sync(0xffffffffu, f1, d);
            if (lane + d < 32) compose2(m00, m01, m10, m11, f0, f1, n00, n01, n10, n11, q0, q1);
        }
        if (lane == 0) {
            double* o = sh + SS::kWarp + 6 * wid;
            o[0] = m00;
            o[1] = m01;
            o[2] = m10;
            o[3] = m11;
            o[4] = f0;
            o[5] = f1;
        }
    }
    __syncthreads();
    SOLVE_MARK(4);
    if (t == 0 && tr.G > 1) {
        double c00 = 1.0, c01 = 0.0, c10 = 0.0, c11 = 1.0, c0 = 0.0, c1 = 0.0;
        for (int w2 = NW - 1; w2 >= 0; --w2) {  // CTA map = W_0 o W_1 o W_2 o W_3
            const double* o = sh + SS::kWarp + 6 * w2;
            double t00 = o[0], t01 = o[1], t10 = o[2], t11 = o[3], t0 = o[4], t1 = o[5];
            compose2(t00, t01, t10, t11, t0, t1, c00, c01, c10, c11, c0, c1);
            c00 = t00;
            c01 = t01;
            c10 = t10;
            c11 = t11;
            c0 = t0;
            c1 = t1;
        }
        double* o = pubb + 6 * tr.rank;
        o[0] = c00;
        o[1] = c01;
        o[2] = c10;
        o[3] = c11;
        o[4] = c0;
        o[5] = c1;
    }
    if (!team_sync(tr.bar, *tr.target, tr.G, tr.err, tr.limit)) return false;
    double* pb = sh + SS::kPub;  // the published back maps of the CTAs after this one
    for (int q = tr.rank + 1 + t; q < tr.G; q += B)
        for (int u = 0; u < 6; ++u) pb[6 * q + u] = __ldcg(&pubb[6 * q + u]);
    __syncthreads();
    // Value folds: a map applied to (s0, s1) gives n_h = fma(M[h][0], s0, fma(M[h][1], s1, f_h))
    // for h = 0, 1.  An FP64 instruction costs the FP64 pipe a whole warp's slot however few of
    // its lanes are active, so each fold runs on a lane pair (lane 2v + h computes n_h of fold v)
    // that swaps its two values by a shuffle: half the instructions of one lane computing both.
    if (t < 2) {  // the boundary values entering each warp, from the CTAs below and the warps
        const int h = t;
        double s0 = 0.0, s1 = 0.0;  // x_n = x_{n+1} = 0 below the last CTA
        for (int q = tr.G - 1; q > tr.rank; --q) {
            const double* o = pb + 6 * q;
            const double nv = fma(o[2 * h], s0, fma(o[2 * h + 1], s1, o[4 + h]));
            const double ov = __shfl_xor_sync(0x3u, nv, 1);
            s0 = h ? ov : nv;
            s1 = h ? nv : ov;
        }
        for (int w2 = NW - 1; w2 >= 0; --w2) {
            sh[SS::kEnter + 2 * w2 + h] = h ? s1 : s0;
            const double* o = sh + SS::kWarp + 6 * w2;
            const double nv = fma(o[2 * h], s0, fma(o[2 * h + 1], s1, o[4 + h]));
            const double ov = __shfl_xor_sync(0x3u, nv, 1);
            s0 = h ? ov : nv;
            s1 = h ? nv : ov;
        }
    }
    __syncthreads();
    // the chunk maps of each warp folded as values, from the warp's boundary values upwards
    // (chunk p receives (x_hi, x_hi+1) in its slots 0 and 1): warp 0 folds 16 warps at once,
    // on the lane pair 2v, 2v + 1 for warp v
    if (wid == 0) {
        const int h = lane & 1;
        for (int v0 = 0; v0 < NW; v0 += 16) {
            const int v = v0 + (lane >> 1);
            const bool on = v < NW;
            double s0 = 0.0, s1 = 0.0;
            if (on) {
                s0 = sh[SS::kEnter + 2 * v];
                s1 = sh[SS::kEnter + 2 * v + 1];
            }
            for (int l = 31; l >= 0; --l) {
                double* o = cm + 6 * (32 * v + l);
                double qa = 0.0, qb = 0.0, qc = 0.0;
                if (on) {
                    qa = o[2 * h];
                    qb = o[2 * h + 1];
                    qc = o[4 + h];
                }
                const double nv = fma(qa, s0, fma(qb, s1, qc));
                __syncwarp();  // both lanes of the pair have read the map before it is overwritten
                if (on) o[h] = h ? s1 : s0;
                const double ov = __shfl_xor_sync(0xffffffffu, nv, 1);
                s0 = h ? ov : nv;
                s1 = h ? nv : ov;
            }
        }
    }
    __syncthreads();
    SOLVE_MARK(5);
    double ysv0 = 0.0, ysv1 = 0.0;  // forward results of rows hi-1, hi-2
    if (act) {
        double cur = cm[6 * t], nxt = cm[6 * t + 1];
        ysv0 = vsm[hi - 1];
        if (hi - 2 >= lo) ysv1 = vsm[hi - 2];
        for (int64_t k = hi - 1; k >= lo; --k) {
            const double y = vsm[k];
            ysave[k] = y;
            const double v = back_row(f.a[k], f.b[k], f.r[k], y, cur, nxt);
            vsm[k] = v;
            if (vout) vout[k] = v;
            nxt = cur;
            cur = v;
        }
    }
    __syncthreads();
    SOLVE_MARK(6);

    // ---------------- consistency at the chunk boundaries ----------------
    // The rows below a CTA's last chunk belong to the next CTA: read them once all are written.
    if (tr.G > 1 && !team_sync(tr.bar, *tr.target, tr.G, tr.err, tr.limit)) return false;
    bool bad = false;
    if (act && hi < n) {
        const double x1 = (hi < r1) ? vsm[hi] : __ldcg(&vout[hi]);
        const double x2 = (hi + 1 >= n) ? 0.0 : ((hi + 1 < r1) ? vsm[hi + 1] : __ldcg(&vout[hi + 1]));
        bad = !row_consistent(f.a[hi - 1], f.b[hi - 1], f.r[hi - 1], ysv0, x1, x2, vsm[hi - 1], tr.tol);
        if (hi - 2 >= lo)
            bad = bad || !row_consistent(f.a[hi - 2], f.b[hi - 2], f.r[hi - 2], ysv1, vsm[hi - 1],
                                         x1, vsm[hi - 2], tr.tol);
    }
    // verdict word: the solve's stamp above the largest failing boundary row (the restart point)
    __shared__ unsigned long long s_top;
    if (t == 0) s_top = 0ull;
    __syncthreads();
    if (bad) atomicMax(&s_top, (unsigned long long)hi);
    bool fallback = __syncthreads_or(bad) != 0;
    SOLVE_MARK(7);
    int64_t top = (int64_t)s_top;
#ifdef TINV_PHASE_PROFILE
    if (bad) {
        // boundary kind: 0 inside a warp, 1 between warps of the CTA, 2 between CTAs
        const int kind = (hi >= r1) ? 2 : (((t + 1) & 31) == 0 ? 1 : 0);
        printf("BADBOUND rank=%d G=%d t=%d hi=%lld kind=%d tol=%g\n", tr.rank, tr.G, t, (long long)hi,
               kind, tr.tol);
    }
#endif
    if (tr.G > 1) {
        if (fallback && t == 0) atomicMax(tr.flag, (tr.stamp << 32) | s_top);
        if (!team_sync(tr.bar, *tr.target, tr.G, tr.err, tr.limit)) return false;
        const unsigned long long v = ld_volatile_u64(tr.flag);
        fallback = (v >> 32) == tr.stamp;
        top = (int64_t)(v & 0xffffffffull);
    }
    if (fallback && tr.G == 1) {
        // one CTA: repair from the failing chunk upwards; the sequential back substitution only
        // for what the repair rounds leave
        const int64_t rest = cta_back_repair(n, f, ysave, vsm, sh, top, L, tr.tol);
        if (rest > 0) {
            staged_seq_back(n, f, ysave, vsm, sh, rest);
            if (t == 0 && tr.nfall) atomicAdd(tr.nfall, 1ull);
        }
        __syncthreads();
        if (vout)
            for (int64_t k = r0 + t; k < r1; k += B) vout[k] = vsm[k];
        __syncthreads();
        return true;
    }
    if (fallback) {
        // the back substitution again, sequentially, by the first CTA of the team, for the rows
        // above the restart point (ysave holds the forward results of all rows)
        if (tr.rank == 0) {
            staged_seq_back(n, f, ysave, tr.G > 1 ? vout : vsm, sh, top);
            if (t == 0 && tr.nfall) atomicAdd(tr.nfall, 1ull);
#ifdef TINV_PHASE_PROFILE
            if (t == 0) printf("FALLBACK G=%d top=%lld n=%lld\n", tr.G, (long long)top, (long long)n);
#endif
        }
        if (tr.G > 1) {
            if (!team_sync(tr.bar, *tr.target, tr.G, tr.err, tr.limit)) return false;
            for (int64_t k = r0 + t; k < r1; k += B) vsm[k] = __ldcg(&vout[k]);
        } else {
            __syncthreads();
            if (vout)
                for (int64_t k = r0 + t; k < r1; k += B) vout[k] = vsm[k];
        }
        __syncthreads();
    }
    return true;
}

// The team solve with 4 chunk warps (the team path; sh holds 2048 doubles, so G <= kTeamMax).
__device__ __forceinline__ bool team_solve(int64_t n, const Fac& f, const double* bsrc, double fac,
                                           double* vsm, double* vout, double* ysave, int64_t r0,
                                           int64_t r1, double* pubf, double* pubb, TeamRef tr,
                                           double* sh)
{
    return team_solve_nw<4>(n, f, bsrc, fac, vsm, vout, ysave, r0, r1, pubf, pubb, tr, sh);
}

enum ColKind { kLower = 0, kUpper = 1 };
enum RowKind { kLowerCol = 0, kUpperCol = 1, kAllCols = 2 };

// Warp-uniform part of per-lane ranges [a, b): lanes that take part pass their range, the
// others (act = false) must not constrain it.
__device__ __forceinline__ void warp_core(int64_t a, int64_t b, bool act, int64_t& lo, int64_t& hi)
{
    int64_t la = act ? a : INT64_MIN, lb = act ? b : INT64_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        la = max(la, __shfl_xor_sync(0xffffffffu, la, o));
        lb = min(lb, __shfl_xor_sync(0xffffffffu, lb, o));
    }
    lo = la;
    hi = lb;
}

// Sum over rows r in [a, b) with r = ph (mod P) of p[r] x[r] (absolute phase), the
// warp-uniform core [lo, hi) (multiples of P) unrolled by 8 with all loads issued first.
template <int P>
__device__ __forceinline__ double dot_phase(const double* __restrict__ p, int64_t st,
                                            const double* x, int64_t a, int64_t b, int64_t lo,
                                            int64_t hi, int ph, bool act)
{
    double acc0 = 0.0, acc1 = 0.0;
    if (!act || b <= a) return 0.0;
    const bool core = lo < hi && lo >= a && hi <= b;
    const int64_t pe = core ? lo : b;
    for (int64_t r = a + ((ph - a) & (P - 1)); r < pe; r += P) acc0 = fma(p[r * st], x[r], acc0);
    if (core) {
        int64_t r = lo + ph;
        for (; r + 7 * P < hi; r += 8 * P) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = p[(r + u * P) * st];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                acc0 = fma(v[u], x[r + u * P], acc0);
                acc1 = fma(v[u + 1], x[r + (u + 1) * P], acc1);
            }
        }
        for (; r < hi; r += P) acc0 = fma(p[r * st], x[r], acc0);
        for (r = hi + ((ph - hi) & (P - 1)); r < b; r += P) acc1 = fma(p[r * st], x[r], acc1);
    }
    return acc0 + acc1;
}

template <int P>
__device__ __forceinline__ void dot2_phase(const double* __restrict__ p, int64_t st,
                                           const double* x, const double* y, int64_t a, int64_t b,
                                           int64_t lo, int64_t hi, int ph, bool act, double& ox,
                                           double& oy)
{
    double ax0 = 0.0, ax1 = 0.0, ay0 = 0.0, ay1 = 0.0;
    ox = oy = 0.0;
    if (!act || b <= a) return;
    const bool core = lo < hi && lo >= a && hi <= b;
    const int64_t pe = core ? lo : b;
    for (int64_t r = a + ((ph - a) & (P - 1)); r < pe; r += P) {
        const double v = p[r * st];
        ax0 = fma(v, x[r], ax0);
        ay0 = fma(v, y[r], ay0);
    }
    if (core) {
        int64_t r = lo + ph;
        for (; r + 7 * P < hi; r += 8 * P) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = p[(r + u * P) * st];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                ax0 = fma(v[u], x[r + u * P], ax0);
                ay0 = fma(v[u], y[r + u * P], ay0);
                ax1 = fma(v[u + 1], x[r + (u + 1) * P], ax1);
                ay1 = fma(v[u + 1], y[r + (u + 1) * P], ay1);
            }
        }
        for (; r < hi; r += P) {
            const double v = p[r * st];
            ax0 = fma(v, x[r], ax0);
            ay0 = fma(v, y[r], ay0);
        }
        for (r = hi + ((ph - hi) & (P - 1)); r < b; r += P) {
            const double v = p[r * st];
            ax1 = fma(v, x[r], ax1);
            ay1 = fma(v, y[r], ay1);
        }
    }
    ox = ax0 + ax1;
    oy = ay0 + ay1;
}

// Warp-uniform core of per-lane ranges, shrunk to multiples of P.
template <int P>
__device__ __forceinline__ void warp_core_al(int64_t a, int64_t b, bool act, int64_t& lo, int64_t& hi)
{
    warp_core(a, b, act, lo, hi);
    lo = (lo + (P - 1)) & ~(int64_t)(P - 1);
    hi = hi & ~(int64_t)(P - 1);
}

// Number of segments 2^lS (lS <= lmax) that minimizes the modelled cost of `groups` warp units
// of `work` FMA instructions per lane, each split into 2^lS pieces: rounds over the nW warps
// times (work per piece + a fixed per-piece overhead) plus the tree levels that add the pieces
// back.  Integer arithmetic only.
__device__ __forceinline__ int pick_segments(int64_t groups, int64_t work, int nW, int lmax)
{
    constexpr int64_t kOvh = 8, kTree = 6;
    int best_l = 0;
    int64_t best = ((groups + nW - 1) / nW) * (work + kOvh);
    for (int l = 1; l <= lmax; ++l) {
        const int64_t units = groups << l;
        const int64_t cost = ((units + nW - 1) / nW) * (((work + (1 << l) - 1) >> l) + kOvh) + kTree * l;
        if (cost < best) {
            best = cost;
            best_l = l;
        }
    }
    return best_l;
}

// Add the S segment partials red[sg*len + c] (c < len, NV values each) by a fixed-shape tree.
__device__ __forceinline__ void tree_segments(double* red, int S, int64_t len, int NV)
{
    // segment stride len*NV <= 2048, so 32-bit indices suffice; segment sg of the lower half
    // takes in segment sg + st
    const int L = (int)(len * NV);
    for (int st = S >> 1; st >= 1; st >>= 1) {
        __syncthreads();
        const int cnt = st * L;
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) red[q] += red[q + st * L];
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// CTA-wide products used by the reorthogonalization.
//
// coldots: out(i, sum_{rho in R(i)} A[rho + i lda] x[rho]) for columns i in [c0, c1), with
//   R(i) = [max(rlo, i), rhi)    (LOWER: the nonzeros of a lower-trapezoidal column), or
//   R(i) = [rlo, min(rhi, i+1))  (UPPER: the nonzeros of an upper-triangular column).
//   A warp takes 8 columns; its lanes are 8 columns x 4 row phases, so each load instruction
//   reads 4 consecutive rows of 8 columns, and the 4 phase partials are added by 2 shuffles.
// rowdots: out(rho, sum_{i in C(rho)} A[rho + i lda] x[i]) for rows rho in [r0, r1), with
//   C(rho) = [0, min(ccap, rho+1))  (LOWERCOL),  [rho, ccap)  (UPPERCOL),  [0, ccap)  (ALL).
//   A warp takes RL = 32, 16 or 8 consecutive rows (fewer rows, more column phases).
// The rows (columns) of the dot products are split into S segments when that fills the warps
// better; segment partials are added by a fixed-shape tree, so results do not depend on
// scheduling.  `red` holds >= 2048 doubles.
// ------------------------------------------------------------------------------------------
template <int KIND, class Out>
__device__ __noinline__ void cta_coldots(const double* __restrict__ A, int64_t lda, int64_t c0, int64_t c1,
                            int64_t rlo, int64_t rhi, const double* x, double* red, Out out)
{
    const int nW = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl = lane >> 2, ph = lane & 3;
    const int64_t nc = c1 - c0;
    if (nc <= 0) return;
    // the rows the columns [c0, c1) can touch (the row segments below are laid over them)
    if (KIND == kLower)
        rlo = max(rlo, c0);
    else
        rhi = min(rhi, c1);
    if (nc <= nW) {
        // few columns: one warp per column, lanes along its rows, one shuffle reduction
        if (wid < nc) {
            const int64_t i = c0 + wid;
            const int64_t a = (KIND == kLower) ? max(rlo, i) : rlo;
            const int64_t b = (KIND == kLower) ? rhi : min(rhi, i + 1);
            const double* p = A + i * lda;
            double acc0 = 0.0, acc1 = 0.0;
            int64_t r = a + lane;
            for (; r + 32 < b; r += 64) {
                acc0 = fma(p[r], x[r], acc0);
                acc1 = fma(p[r + 32], x[r + 32], acc1);
            }
            if (r < b) acc0 = fma(p[r], x[r], acc0);
            const double v = warp_sum(acc0 + acc1);
            if (lane == 0) out(i, v);
        }
        __syncthreads();
        return;
    }
    const int64_t groups = (nc + 7) / 8;
    const int64_t rows = rhi > rlo ? rhi - rlo : 0;
    int lmax = 0;  // S = 2^lS row segments, each >= 32 rows, partials fit in red
    while (lmax < 4 && ((int64_t)nc << (lmax + 1)) <= 2048 && rows >= ((int64_t)32 << (lmax + 1))) ++lmax;
    const int lS = pick_segments(groups, (rows + 3) / 4, nW, lmax);
    const int S = 1 << lS;
    const int64_t seglen = (rows + S - 1) >> lS;
    const int64_t units = groups << lS;
    for (int64_t u = wid; u < units; u += nW) {
        const int64_t g = u >> lS;
        const int sg = (int)(u & (S - 1));
        const int64_t i = c0 + g * 8 + cl;
        const bool act = i < c1;
        const int64_t s_lo = rlo + sg * seglen, s_hi = min(rhi, s_lo + seglen);
        int64_t a = 0, b = 0;
        if (act) {
            a = max(s_lo, (KIND == kLower) ? max(rlo, i) : rlo);
            b = min(s_hi, (KIND == kLower) ? rhi : min(rhi, i + 1));
            if (b < a) b = a;
        }
        int64_t lo, hi;
        warp_core_al<4>(a, b, act && a < b, lo, hi);
        double v = dot_phase<4>(A + (act ? i : c0) * lda, 1, x, a, b, lo, hi, ph, act);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (act && ph == 0) {
            if (S == 1)
                out(i, v);
            else
                red[(int64_t)sg * nc + (i - c0)] = v;
        }
    }
    if (S > 1) {
        tree_segments(red, S, nc, 1);
        for (int64_t c = threadIdx.x; c < nc; c += blockDim.x) out(c0 + c, red[c]);
    }
    __syncthreads();
}

template <int RL, int KIND, int NV, class Out>
__device__ __noinline__ void rowdots_rl(const double* __restrict__ A, int64_t lda, int64_t r0, int64_t r1,
                           int64_t ccap, const double* x0, const double* x1, double* red, Out out)
{
    constexpr int CL = 32 / RL;
    const int nW = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rr = lane % RL, ph = lane / RL;
    const int64_t nr = r1 - r0;
    const int64_t rgroups = (nr + RL - 1) / RL;
    // fixed column grid over the columns any row of [r0, r1) can touch
    const int64_t gb = (KIND == kUpperCol) ? r0 : 0;
    const int64_t ge = (KIND == kLowerCol) ? min(ccap, r1) : ccap;
    const int64_t glen = ge > gb ? ge - gb : 0;
    int lmax = 0;  // S = 2^lS column segments, each >= 8 CL columns, partials fit in red
    while (lmax < 5 && ((int64_t)nr * NV << (lmax + 1)) <= 2048 && glen >= ((int64_t)8 * CL << (lmax + 1))) ++lmax;
    const int lS = pick_segments(rgroups, (glen + CL - 1) / CL * NV, nW, lmax);
    const int S = 1 << lS;
    const int64_t seglen = (glen + S - 1) >> lS;
    const int64_t units = rgroups << lS;
    for (int64_t u = wid; u < units; u += nW) {
        const int64_t g = u >> lS;
        const int sg = (int)(u & (S - 1));
        const int64_t rho = r0 + g * RL + rr;
        const bool act = rho < r1;
        int64_t a = 0, b = 0;
        if (act) {
            const int64_t s0 = gb + sg * seglen, s1 = min(ge, s0 + seglen);
            const int64_t cb = (KIND == kUpperCol) ? rho : 0;
            const int64_t ce = (KIND == kLowerCol) ? min(ccap, rho + 1) : ccap;
            a = max(s0, cb);
            b = min(s1, ce);
            if (b < a) b = a;
        }
        int64_t lo, hi;
        warp_core_al<CL>(a, b, act && a < b, lo, hi);
        double v0, v1 = 0.0;
        const double* prow = A + (act ? rho : r0);
        if (NV == 2)
            dot2_phase<CL>(prow, lda, x0, x1, a, b, lo, hi, ph, act, v0, v1);
        else
            v0 = dot_phase<CL>(prow, lda, x0, a, b, lo, hi, ph, act);
#pragma unroll
        for (int o = RL; o < 32; o <<= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            if (NV == 2) v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        }
        if (act && ph == 0) {
            if (S == 1) {
                out(rho, v0, v1);
            } else {
                red[((int64_t)sg * nr + (rho - r0)) * NV] = v0;
                if (NV == 2) red[((int64_t)sg * nr + (rho - r0)) * NV + 1] = v1;
            }
        }
    }
    if (S > 1) {
        tree_segments(red, S, nr, NV);
        for (int64_t q = threadIdx.x; q < nr; q += blockDim.x)
            out(r0 + q, red[q * NV], (NV == 2) ? red[q * NV + 1] : 0.0);
    }
    __syncthreads();
}

template <int KIND, int NV, class Out>
__device__ void cta_rowdots(const double* __restrict__ A, int64_t lda, int64_t r0, int64_t r1,
                            int64_t ccap, const double* x0, const double* x1, double* red, Out out)
{
    const int64_t nr = r1 - r0;
    if (nr <= 0) return;
    const int nW = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (nr <= nW) {
        // few rows: one warp per row, lanes along its columns, one shuffle reduction
        if (wid < nr) {
            const int64_t rho = r0 + wid;
            const int64_t a = (KIND == kUpperCol) ? rho : 0;
            const int64_t b = (KIND == kLowerCol) ? min(ccap, rho + 1) : ccap;
            const double* p = A + rho;
            double s0 = 0.0, s1 = 0.0;
            for (int64_t i = a + lane; i < b; i += 32) {
                const double v = p[i * lda];
                s0 = fma(v, x0[i], s0);
                if (NV == 2) s1 = fma(v, x1[i], s1);
            }
            s0 = warp_sum(s0);
            if (NV == 2) s1 = warp_sum(s1);
            if (lane == 0) out(rho, s0, s1);
        }
        __syncthreads();
        return;
    }
    if (nr > 16)
        rowdots_rl<32, KIND, NV>(A, lda, r0, r1, ccap, x0, x1, red, out);
    else if (nr > 8)
        rowdots_rl<16, KIND, NV>(A, lda, r0, r1, ccap, x0, x1, red, out);
    else
        rowdots_rl<8, KIND, NV>(A, lda, r0, r1, ccap, x0, x1, red, out);
}

}  // namespace tinvx
