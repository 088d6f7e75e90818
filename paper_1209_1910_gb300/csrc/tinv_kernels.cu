// tinv_kernels.cu -- sm_103a kernels of libtinv.
//
//   k_plan_seg : one CTA per problem: ||T||_1, cluster tolerance, DSTEIN shift perturbation
//                (Sec. 2.1; Alg. 4).
//   k_plan_list: Peters-Wilkinson cluster heads over all problems (Alg. 4), cluster
//                list, T offsets and the assignment of clusters to CTA teams of the persistent
//                kernel (large clusters) or to its work queue (the rest, largest first).
//   k_lu     : one thread per shift: LU with scaled partial pivoting of T - s_j I (Eq. 1).
//   k_first  : one warp per eigenvalue: random start, DSTEIN scaling and the chunked solve; full
//              sweep loop + normalization for cluster heads and singletons (Alg. 1 / Alg. 4
//              without reorthogonalization), first sweep only for the other cluster members.
//   k_chain  : persistent cooperative kernel: each cluster's members in order (Alg. 4 j-loop),
//              with the compact-WY update of Sec. 3.3.2 spread over a team of CTAs (or MGS,
//              Alg. 1, on one CTA per cluster).
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>

#include "tinv_device.cuh"

namespace tinvx {

// ==========================================================================================
// Plan
// ==========================================================================================

// Inclusive block scans over blockDim (multiple of 32) values; sred >= 33 entries.
template <typename TV, class Op>
__device__ TV block_scan_incl(TV v, TV* sred, Op op, TV ident, TV* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        TV u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = op(u, v);
    }
    __syncthreads();
    if (lane == 31) sred[wid] = v;
    __syncthreads();
    if (wid == 0) {
        TV s = lane < nw ? sred[lane] : ident;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            TV u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s = op(u, s);
        }
        sred[lane] = s;  // inclusive prefix of warp totals
    }
    __syncthreads();
    if (wid > 0) v = op(sred[wid - 1], v);
    *total = sred[nw - 1];
    __syncthreads();
    return v;
}

struct OpMax {
    template <typename T>
    __device__ T operator()(T a, T b) const { return a > b ? a : b; }
};
struct OpAdd {
    template <typename T>
    __device__ T operator()(T a, T b) const { return a + b; }
};

// ||T||_1 = max_i (|d_i| + |e_{i-1}|) + |e_i|   (added in this order, as the oracle)
__device__ double block_onenorm(int64_t n, const double* d, const double* e, double* sredd)
{
    double loc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double s = fabs(d[i]);
        if (i > 0) s = __dadd_rn(s, fabs(e[i - 1]));
        if (i < n - 1) s = __dadd_rn(s, fabs(e[i]));
        loc = fmax(loc, s);
    }
    return block_max(loc, sredd);
}

// Norm and tolerances of a single problem (the stand-alone solve): w.scal and the counters.
__global__ void __launch_bounds__(kPlanThreads) k_norm(Problem p, Ws w)
{
    __shared__ double sredd[33];
    const double onenrm = block_onenorm(p.n, p.d, p.e, sredd);
    if (threadIdx.x == 0) {
        w.scal[0] = onenrm;
        w.scal[1] = __dmul_rn(1e-3, onenrm);
        w.scal[2] = __dsqrt_rn(__ddiv_rn(0.1, (double)p.n));
        w.scal[3] = 0.0;
        for (int c = 0; c < kCtrCount; ++c) w.ctr[c] = 0;
    }
}

// Plan, part 1: one CTA per problem.  ||T||_1, the cluster tolerance, the convergence threshold
// (Sec. 2.1; Alg. 4), the problem index of each eigenvalue and the DSTEIN shift
// perturbation: if w_j - w'_{j-1} < 10 eps |w_j| then w'_j = w'_{j-1} + 10 eps |w_j|.
__global__ void __launch_bounds__(kPlanThreads) k_plan_seg(Problem p, Ws w)
{
    __shared__ double sredd[33];
    __shared__ int s_tight;
    const int t = threadIdx.x, B = blockDim.x;
    const int32_t sidx = blockIdx.x;
    if (!p.seg_preset) {
        if (t == 0) {
            Seg g;
            memset(&g, 0, sizeof(g));
            g.n = p.n;
            g.m = p.m;
            g.ldz = p.ldz;
            g.kj0 = p.j0;
            g.seed = p.seed;
            w.segs[0] = g;
        }
        __syncthreads();
    }
    const Seg g = w.segs[sidx];
    const int64_t n = g.n, m = g.m;
    const double* d = p.d + g.de;
    const double* e = p.e + g.de;
    const double* wv = p.w + g.wo;
    const double onenrm = n > 0 ? block_onenorm(n, d, e, sredd) : 0.0;
    const double ortol = __dmul_rn(1e-3, onenrm);
    const double dtpcrt = n > 0 ? __dsqrt_rn(__ddiv_rn(0.1, (double)n)) : 0.0;
    if (t == 0) {
        w.segs[sidx].onenrm = onenrm;
        w.segs[sidx].ortol = ortol;
        w.segs[sidx].dtpcrt = dtpcrt;
        w.sinfo[sidx] = 0;
        s_tight = 0;
        if (sidx == 0) {
            w.scal[0] = onenrm;
            w.scal[1] = ortol;
            w.scal[2] = dtpcrt;
            w.scal[3] = 0.0;
            for (int c = 0; c < kCtrCount; ++c) w.ctr[c] = 0;
        }
    }
    if (sidx == 0) {
        for (int b = t; b < w.P; b += B) w.bar[b] = 0u;
        if (w.partScal)  // the teams' consistency-verdict words (slot 15 of each block)
            for (int b = t; b < w.P; b += B)
                ((unsigned long long*)w.partScal)[(size_t)b * kScalTeam + 15] = 0ull;
    }
    for (int64_t jl = t; jl < m; jl += B) w.segj[g.j0 + jl] = sidx;
    __syncthreads();
    // without any tight pair w' = w; otherwise one thread scans
    for (int64_t j = 1 + t; j < m; j += B) {
        const double xj = wv[j];
        const double pertol = __dmul_rn(10.0, fabs(__dmul_rn(kEps, xj)));
        if (__dsub_rn(xj, wv[j - 1]) < pertol) s_tight = 1;
    }
    __syncthreads();
    double* wp = w.wp + g.j0;
    if (s_tight == 0) {
        for (int64_t j = t; j < m; j += B) wp[j] = wv[j];
    } else if (t == 0) {
        double xjm = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            double xj = wv[j];
            if (j > 0) {
                const double pertol = __dmul_rn(10.0, fabs(__dmul_rn(kEps, xj)));
                if (__dsub_rn(xj, xjm) < pertol) xj = __dadd_rn(xjm, pertol);
            }
            wp[j] = xj;
            xjm = xj;
        }
    }
}

// Peters-Wilkinson test on consecutive perturbed shifts of one problem (Sec. 2.1): a new cluster
// starts at the problem's first eigenvalue or after a gap larger than 1e-3 ||T||_1.
__device__ __forceinline__ bool new_cluster(const Ws& w, int64_t j)
{
    const Seg* g = w.segs + w.segj[j];
    return j == g->j0 || fabs(__dsub_rn(w.wp[j], w.wp[j - 1])) > g->ortol;
}

// Work of one cluster (flops of its reorthogonalization grow as size^2 n) and the team-size cap.
__device__ __forceinline__ double cluster_work(const Ws& w, int32_t c)
{
    const double sz = (double)w.clsize[c];
    return sz * sz * (double)w.segs[w.segj[w.clstart[c]]].n;
}

constexpr int kMaxCand = 1024;   // team candidates: at most P / 2 <= 1024
constexpr int kSliceTeam = 32;  // teams at least this large reduce s and g by slices

// Plan, part 2: one CTA over all eigenvalues.  Cluster heads and the list of clusters with >= 2
// members, T offsets, and the assignment of clusters to CTA teams of the persistent kernel:
// clusters whose share of the work is worth >= 2 CTAs get a contiguous team; the rest form a
// queue, largest first, served by single CTAs (also by team CTAs once their cluster is done).
__global__ void __launch_bounds__(kPlanThreads) k_plan_list(Problem p, Ws w, int32_t max_team)
{
    __shared__ double sredd[33];
    __shared__ int32_t sredi[33];
    __shared__ int64_t sredl[33];
    __shared__ int32_t s_cand[kMaxCand];
    __shared__ uint8_t s_team[kMaxCand];
    __shared__ int32_t s_gsz[kMaxCand];
    __shared__ int32_t s_hist[64], s_cur[64];
    __shared__ int32_t s_ncand;
    const int t = threadIdx.x, B = blockDim.x;
    const int64_t M = p.M;
    const int32_t P = w.P;

    // heads (max-scan of head positions); a start is a head whose successor continues its
    // cluster, an end is a member whose successor is a head (or the last index)
    int32_t carry_head = 0, carry_cnt = 0, carry_end = 0;
    for (int64_t base = 0; base < M; base += B) {
        const int64_t j = base + t;
        const bool in = j < M;
        const bool fj = in && new_cluster(w, j);
        const bool fj1 = in && (j + 1 < M) && new_cluster(w, j + 1);
        const bool is_start = fj && (j + 1 < M) && !fj1;
        const bool is_end = in && !fj && (j + 1 == M || fj1);
        int32_t tot, tot2, tot3;
        int32_t hd = block_scan_incl<int32_t>(fj ? (int32_t)j : 0, sredi, OpMax(), 0, &tot);
        hd = max(hd, carry_head);
        const int32_t cs = block_scan_incl<int32_t>(is_start ? 1 : 0, sredi, OpAdd(), 0, &tot2);
        const int32_t ce = block_scan_incl<int32_t>(is_end ? 1 : 0, sredi, OpAdd(), 0, &tot3);
        if (in) w.head[j] = hd;
        if (is_start) w.clstart[carry_cnt + cs - 1] = (int32_t)j;
        if (is_end) w.clsize[carry_end + ce - 1] = (int32_t)(j - hd + 1);
        carry_head = max(carry_head, tot);
        carry_cnt += tot2;
        carry_end += tot3;
        __syncthreads();
    }
    const int32_t K = carry_cnt;
    __syncthreads();
    // T offsets: exclusive prefix sum of size^2
    int64_t carry_off = 0;
    for (int64_t base = 0; base < K; base += B) {
        const int64_t c = base + t;
        const int64_t sz = (c < K) ? (int64_t)w.clsize[c] : 0;
        int64_t tot;
        int64_t inc = block_scan_incl<int64_t>(sz * sz, sredl, OpAdd(), (int64_t)0, &tot);
        if (c < K) w.cltoff[c] = carry_off + inc - sz * sz;
        carry_off += tot;
        __syncthreads();
    }
    for (int32_t b = t; b < P; b += B) {
        w.sched[4 * b + 0] = b;
        w.sched[4 * b + 1] = 1;
        w.sched[4 * b + 2] = 0;
        w.sched[4 * b + 3] = -1;
    }
    if (t < 64) s_hist[t] = 0;
    if (t == 0) {
        w.ctr[kCtrNClust] = K;
        w.ctr[kCtrTSize] = carry_off;
        s_ncand = 0;
    }
    __syncthreads();

    // team candidates (MGS and single-CTA grids use the queue only)
    double wl = 0.0;
    for (int32_t c = t; c < K; c += B) wl += cluster_work(w, c);
    const double wtot = block_sum(wl, sredd);
    const bool teams = (p.method == 0) && P >= 2 && K > 0;
    int32_t carry_c = 0;
    for (int32_t base = 0; base < K; base += B) {
        const int32_t c = base + t;
        bool cand = false;
        if (teams && c < K) {
            const double wc = cluster_work(w, c);
            int64_t gmax = min((int64_t)min(P, kTeamMax), max((int64_t)1, w.segs[w.segj[w.clstart[c]]].n / 16));
            if (max_team > 0) gmax = min(gmax, (int64_t)max_team);
            cand = floor((double)P * wc / wtot) >= 2.0 && gmax >= 2;
        }
        int32_t tot;
        const int32_t pos = block_scan_incl<int32_t>(cand ? 1 : 0, sredi, OpAdd(), 0, &tot);
        if (cand && carry_c + pos - 1 < kMaxCand) s_cand[carry_c + pos - 1] = c;
        carry_c += tot;
        __syncthreads();
    }
    const int32_t ncand = min(carry_c, kMaxCand);
    if (t == 0) {
        double wteam = 0.0;
        for (int32_t i = 0; i < ncand; ++i) wteam += cluster_work(w, s_cand[i]);
        const double wq = wtot - wteam;
        int32_t Q = 0;
        if (wq > 0.0) Q = max(1, (int32_t)llrint(P * wq / wtot));
        const int32_t Pteam = max(0, P - Q);
        // team sizes: floor of each candidate's share; the CTAs left over go one each to the
        // teams with the largest fractional shares (ties to the earlier cluster)
        int32_t used = 0;
        for (int32_t i = 0; i < ncand; ++i) {
            const int32_t c = s_cand[i];
            int32_t gmax = (int32_t)min((int64_t)min(P, kTeamMax), max((int64_t)1, w.segs[w.segj[w.clstart[c]]].n / 16));
            if (max_team > 0) gmax = min(gmax, max_team);
            const double share = Pteam * cluster_work(w, c) / wteam;
            const int32_t g = min(gmax, (int32_t)floor(share));
            s_gsz[i] = g;
            if (g >= 2) used += g;
        }
        for (int32_t left = Pteam - used; left > 0; --left) {
            int32_t best = -1;
            double bf = -1.0;
            for (int32_t i = 0; i < ncand; ++i) {
                const int32_t c = s_cand[i];
                int32_t gmax = (int32_t)min((int64_t)min(P, kTeamMax), max((int64_t)1, w.segs[w.segj[w.clstart[c]]].n / 16));
                if (max_team > 0) gmax = min(gmax, max_team);
                if (s_gsz[i] < 2 || s_gsz[i] >= gmax) continue;
                const double share = Pteam * cluster_work(w, c) / wteam;
                const double fr = share - (double)s_gsz[i];
                if (fr > bf) {
                    bf = fr;
                    best = i;
                }
            }
            if (best < 0) break;
            ++s_gsz[best];
        }
        int32_t next = 0;
        for (int32_t i = 0; i < ncand; ++i) {
            const int32_t c = s_cand[i];
            const int32_t g = s_gsz[i];
            s_team[i] = 0;
            if (g >= 2 && next + g <= Pteam) {
                for (int32_t r = 0; r < g; ++r) {
                    const int32_t b = next + r;
                    w.sched[4 * b + 0] = next;
                    w.sched[4 * b + 1] = g;
                    w.sched[4 * b + 2] = r;
                    w.sched[4 * b + 3] = c;
                }
                next += g;
                s_team[i] = 1;
            }
        }
        s_ncand = ncand;
    }
    __syncthreads();

    // queue: every cluster without a team, in decreasing order of work (buckets of powers of 2)
    auto on_team = [&](int32_t c) {
        for (int32_t i = 0; i < s_ncand; ++i)
            if (s_cand[i] == c) return s_team[i] != 0;
        return false;
    };
    auto bucket = [&](int32_t c) { return 63 - min(63, max(0, ilogb(cluster_work(w, c)))); };
    for (int32_t c = t; c < K; c += B)
        if (!on_team(c)) atomicAdd(&s_hist[bucket(c)], 1);
    __syncthreads();
    if (t == 0) {
        int32_t acc = 0;
        for (int i = 0; i < 64; ++i) {
            s_cur[i] = acc;
            acc += s_hist[i];
        }
        w.ctr[kCtrNQueue] = acc;
        w.ctr[kCtrQHead] = 0;
    }
    __syncthreads();
    for (int32_t c = t; c < K; c += B)
        if (!on_team(c)) w.queue[atomicAdd(&s_cur[bucket(c)], 1)] = c;
}

// Plan for stand-alone orthogonalization: one problem, one cluster made of all m columns.
__global__ void k_orth_plan(Problem p, Ws w, int32_t method)
{
    const int t = threadIdx.x;
    for (int b = t; b < w.P; b += blockDim.x) {
        w.bar[b] = 0u;
        w.sched[4 * b + 0] = b;
        w.sched[4 * b + 1] = 1;
        w.sched[4 * b + 2] = 0;
        w.sched[4 * b + 3] = -1;
    }
    for (int64_t j = t; j < p.m; j += blockDim.x) w.segj[j] = 0;
    if (t == 0) {
        Seg g;
        memset(&g, 0, sizeof(g));
        g.n = p.n;
        g.m = p.m;
        g.ldz = p.ldz;
        w.segs[0] = g;
        for (int c = 0; c < kCtrCount; ++c) w.ctr[c] = 0;
        w.clstart[0] = 0;
        w.clsize[0] = (int32_t)p.m;
        w.cltoff[0] = 0;
        w.ctr[kCtrNClust] = 1;
        w.ctr[kCtrTSize] = p.m * p.m;
        w.scal[0] = w.scal[1] = w.scal[2] = w.scal[3] = 0.0;
    }
    __syncthreads();
    if (t == 0) {
        if (method == 0 && w.P >= 2) {
            const int32_t g = w.P;
            for (int32_t r = 0; r < g; ++r) {
                w.sched[4 * r + 0] = 0;
                w.sched[4 * r + 1] = g;
                w.sched[4 * r + 2] = r;
                w.sched[4 * r + 3] = 0;
            }
            w.ctr[kCtrNQueue] = 0;
        } else {
            w.queue[0] = 0;
            w.ctr[kCtrNQueue] = 1;
        }
    }
}

// ==========================================================================================
// LU of T - s I with scaled partial pivoting, one thread per shift (bit-exact: explicit
// round-to-nearest operations, no contraction).  Row j of each output holds shift j.
// ==========================================================================================

// Interchange decision of the scaled pivoting rule: true iff fl(|c|/s2) > fl(|a|/s1) (the rule
// written with correctly rounded quotients; a zero numerator counts as 0).  All four arguments
// are non-negative, and non-negative doubles are ordered as their bit patterns, so the tests
// below are integer compares (they stay off the FP64 pipe, whose latency bounds this
// one-thread-per-shift recurrence).  Most steps are decided from the cross products P = |c| s1
// and Q = |a| s2: when both are normal and their bit patterns differ by more than 16, the larger
// exceeds the smaller by at least 17 units in the last place of the smaller, more than a
// relative 2^-49, and then the rounded quotients are ordered the same way (each quotient and
// product carries at most 2^-53 relative rounding error).  Only inside that band, or when a
// product is not normal, are the two divisions evaluated.
__device__ __forceinline__ bool lu_interchange(double aa, double s1, double cc, double s2)
{
    if (__double_as_longlong(cc) == 0) return false;
    if (__double_as_longlong(aa) == 0) return true;
    const long long P = __double_as_longlong(__dmul_rn(cc, s1));  // |c| s1
    const long long Q = __double_as_longlong(__dmul_rn(aa, s2));  // |a| s2
    constexpr long long kMinNormal = 0x0010000000000000ll;         // DBL_MIN
    constexpr long long kLarge = 0x7e37e43c8800759cll;             // 1e300
    if (P >= kMinNormal && Q >= kMinNormal && P <= kLarge && Q <= kLarge) {
        if (P > Q + 16) return true;
        if (Q > P + 16) return false;
    }
    return __ddiv_rn(cc, s2) > __ddiv_rn(aa, s1);
}

__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// LU of T - lam I (order n) into one row of each output; |u_nn| and the tiny-pivot threshold
// eps max|U| (eps if U = 0) go to *u0n and *tolv when those are given.
__device__ __forceinline__ void lu_row(int64_t n, const double* __restrict__ d,
                                       const double* __restrict__ e, double lam, double* __restrict__ l,
                                       double* __restrict__ u0, double* __restrict__ u1,
                                       double* __restrict__ u2, uint8_t* __restrict__ pv,
                                       double* u0n, double* tolv)
{
    double ak = __dsub_rn(d[0], lam);
    double bk = (n > 1) ? e[0] : 0.0;
    unsigned long long umax = 0;  // max |U entry| as the bit pattern of a non-negative double
    for (int64_t k = 0; k + 1 < n; ++k) {
        const double ck = e[k];
        const double a1 = __dsub_rn(d[k + 1], lam);
        const double b1 = (k + 2 < n) ? e[k + 1] : 0.0;
        const double scale1 = __dadd_rn(fabs(ak), fabs(bk));
        const double scale2 = __dadd_rn(__dadd_rn(fabs(ck), fabs(a1)), fabs(b1));
        double lk, w0, w1, w2;
        uint8_t sw;
        if (!lu_interchange(fabs(ak), scale1, fabs(ck), scale2)) {
            lk = (ck == 0.0) ? 0.0 : __ddiv_rn(ck, ak);
            w0 = ak;
            w1 = bk;
            w2 = 0.0;
            sw = 0;
            ak = __dsub_rn(a1, __dmul_rn(lk, bk));
            bk = b1;
        } else {
            lk = __ddiv_rn(ak, ck);
            w0 = ck;
            w1 = a1;
            w2 = b1;
            sw = 1;
            ak = __dsub_rn(bk, __dmul_rn(lk, a1));
            bk = -__dmul_rn(lk, b1);
        }
        l[k] = lk;
        u0[k] = w0;
        u1[k] = w1;
        u2[k] = w2;
        pv[k] = sw;
        umax = max(umax, max(abs_bits(w0), max(abs_bits(w1), abs_bits(w2))));
    }
    u0[n - 1] = ak;
    l[n - 1] = 0.0;
    u1[n - 1] = 0.0;
    u2[n - 1] = 0.0;
    pv[n - 1] = 0;
    umax = max(umax, abs_bits(ak));
    if (u0n) *u0n = fabs(ak);
    if (tolv) {
        double tol = __dmul_rn(kEps, __longlong_as_double((long long)umax));
        if (tol == 0.0) tol = kEps;
        *tolv = tol;
    }
}

// One problem, shift j in row j (stride n) of every output (tinv_lu, tinv_solve).
__global__ void k_lu(int64_t n, const double* __restrict__ d, const double* __restrict__ e,
                     int64_t m, const double* __restrict__ shift, double* __restrict__ L,
                     double* __restrict__ U0, double* __restrict__ U1, double* __restrict__ U2,
                     uint8_t* __restrict__ PV, double* __restrict__ u0n, double* __restrict__ tolv)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const size_t base = (size_t)j * (size_t)n;
    lu_row(n, d, e, shift[j], L + base, U0 + base, U1 + base, U2 + base, PV + base,
           u0n ? u0n + j : nullptr, tolv ? tolv + j : nullptr);
}

// Problem table: global eigenvalue j of problem s, shift w'_j, rows at the problem's offsets.
__global__ void k_lu_seg(Problem p, Ws w, int lanes)
{
    if ((int)threadIdx.x >= lanes) return;
    const int64_t j = (int64_t)blockIdx.x * lanes + threadIdx.x;
    if (j >= p.M) return;
    const Seg* g = w.segs + w.segj[j];
    const int64_t n = g->n;
    const size_t base = (size_t)(g->foff + (j - g->j0) * n);
    if (!TINV_IN(j < w.nM && dbg_range((int64_t)base, (int64_t)base + n, w.nF), (int*)&w.ctr[kCtrErr]))
        return;
    lu_row(n, p.d + g->de, p.e + g->de, w.wp[j], w.fl + base, w.fr + base, w.fu1 + base,
           w.fu2 + base, w.fpiv + base, w.u0n + j, w.tolv + j);
}

// Solve-ready back-substitution factors, in place: r = 1/u0, a = -u1 r, b = -u2 r.  A pivot so
// small that one of these quotients could overflow, |u0| < DBL_MIN max(1, |u1|, |u2|) (zero
// included), is replaced by sign(u0) tol (sign(0) = +, tol = eps max|U|): the perturbation
// DLAGTS makes only to avoid overflow, decided on U alone so that the back substitution stays a
// fixed linear recurrence.
__device__ __forceinline__ void recip_row(int64_t n, double* __restrict__ u0, double* __restrict__ u1,
                                          double* __restrict__ u2, double tol)
{
    constexpr double kDblMin = 2.2250738585072014e-308;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        double a = u0[k];
        const double big = fmax(1.0, fmax(fabs(u1[k]), fabs(u2[k])));
        if (fabs(a) < __dmul_rn(kDblMin, big)) a = (a >= 0.0) ? tol : -tol;
        const double r = __drcp_rn(a);
        u0[k] = r;
        u1[k] = -u1[k] * r;
        u2[k] = -u2[k] * r;
    }
}

__global__ void k_recip(int64_t n, int64_t m, double* __restrict__ U0R, double* __restrict__ U1,
                        double* __restrict__ U2, const double* __restrict__ tolv)
{
    for (int64_t j = blockIdx.x; j < m; j += gridDim.x) {
        const size_t o = (size_t)j * (size_t)n;
        recip_row(n, U0R + o, U1 + o, U2 + o, tolv[j]);
    }
}

__global__ void k_recip_seg(Problem p, Ws w)
{
    for (int64_t j = blockIdx.x; j < p.M; j += gridDim.x) {
        const Seg* g = w.segs + w.segj[j];
        const size_t o = (size_t)(g->foff + (j - g->j0) * g->n);
        if (!TINV_IN(dbg_range((int64_t)o, (int64_t)o + g->n, w.nF), (int*)&w.ctr[kCtrErr])) return;
        recip_row(g->n, w.fr + o, w.fu1 + o, w.fu2 + o, w.tolv[j]);
    }
}

// ==========================================================================================
// One warp per eigenvalue: start vector, DSTEIN scaling, chunked solve, convergence test and
// normalization (cluster heads and singletons); cluster members get their first solve only.
// ==========================================================================================
__device__ __forceinline__ Fac fac_at(const Ws& w, size_t base)
{
    Fac f;
    f.l = w.fl + base;
    f.a = w.fu1 + base;  // -u1/u0 after k_recip
    f.b = w.fu2 + base;  // -u2/u0
    f.r = w.fr + base;
    f.piv = w.fpiv + base;
    return f;
}

// Factor rows of eigenvalue j of a single problem of order n (stand-alone solve).
__device__ __forceinline__ Fac fac_of(const Ws& w, int64_t j, int64_t n)
{
    return fac_at(w, (size_t)j * (size_t)n);
}

// Global eigenvalue j of the problem table: its problem, local index and factor-row offset.
struct JRef {
    const Seg* g;
    int64_t jl;
    size_t off;
};
__device__ __forceinline__ JRef jref(const Ws& w, int64_t j)
{
    JRef r;
    r.g = w.segs + w.segj[j];
    r.jl = j - r.g->j0;
    r.off = (size_t)(r.g->foff + r.jl * r.g->n);
    return r;
}

__device__ void warp_scale(int64_t n, double* x, double onenrm, double u0n, int lane)
{
    double as = 0.0;
    for (int64_t i = lane; i < n; i += 32) as += fabs(x[i]);
    as = warp_sum(as);
    const double scl = ((double)n * onenrm) * fmax(kEps, u0n) / as;
    __syncwarp();
    for (int64_t i = lane; i < n; i += 32) x[i] *= scl;
    __syncwarp();
}

// Record a vector that did not converge (total and per problem).
__device__ __forceinline__ void count_nonconverged(const Ws& w, int64_t j)
{
    atomicAdd((unsigned long long*)&w.ctr[kCtrInfo], 1ull);
    atomicAdd((unsigned long long*)&w.sinfo[w.segj[j]], 1ull);
}

__global__ void __launch_bounds__(kFirstWarps * 32) k_first(Problem p, Ws w)
{
    __shared__ double sh_all[kFirstWarps][8 * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kFirstWarps + warp;
    if (j >= p.M) return;
    double* sh = sh_all[warp];
    const JRef jr = jref(w, j);
    const Seg& g = *jr.g;
    const int64_t n = g.n;
    double* x = p.Z + g.z + jr.jl * g.ldz;
    if (!TINV_IN(dbg_range((int64_t)jr.off, (int64_t)jr.off + n, w.nF) &&
                     (p.zlen == 0 || dbg_range(g.z + jr.jl * g.ldz, g.z + jr.jl * g.ldz + n, p.zlen)),
                 (int*)&w.ctr[kCtrErr]))
        return;
    const Fac f = fac_at(w, jr.off);
    const double onenrm = g.onenrm, dtpcrt = g.dtpcrt, u0n = w.u0n[j];
    const bool is_head = (w.head[j] == (int32_t)j);
    if (n == 1) {  // T = [d_1]: z = [1]
        if (lane == 0) {
            x[0] = 1.0;
            if (p.iters) p.iters[j] = 1;
        }
        return;
    }
    const uint64_t key = start_key(g.seed, g.kj0 + jr.jl, 0);
    for (int64_t i = lane; i < n; i += 32) x[i] = start_value(key, i);
    __syncwarp();
    const int maxits = is_head ? kMaxIts : 1;
    int nrmchk = 0, its = 0;
    bool conv = false;
    double* ysave = w.Y + jr.off;  // free until the cluster kernel writes this Y column
    while (its < maxits) {
        ++its;
        warp_scale(n, x, onenrm, u0n, lane);
        // a member's first sweep only starts the cluster kernel's sweeps; a head's sweep can
        // be its last once it has kExtra successes or reaches the sweep limit
        const bool may_end = is_head && (nrmchk >= kExtra || its == maxits);
        if (chunk_solve(n, f, x, ysave, sh, lane, 32, WarpSync(), may_end ? kSolveTol : kSolveTolLoose) &&
            lane == 0)
            atomicAdd((unsigned long long*)&w.ctr[kCtrFallbackFirst], 1ull);
        if (!is_head) break;
        double mx = 0.0;
        for (int64_t i = lane; i < n; i += 32) mx = fmax(mx, fabs(x[i]));
        mx = warp_max(mx);
        if (mx >= dtpcrt && ++nrmchk >= kExtra + 1) {
            conv = true;
            break;
        }
    }
    if (!is_head) return;
    // normalize; the first entry of largest magnitude becomes positive
    double ss = 0.0, am = -1.0;
    int64_t ai = 0;
    for (int64_t i = lane; i < n; i += 32) {
        const double v = x[i];
        ss = fma(v, v, ss);
        if (fabs(v) > am) {
            am = fabs(v);
            ai = i;
        }
    }
    ss = warp_sum(ss);
    warp_argmax(am, ai);
    double s = 1.0 / sqrt(ss);
    if (x[ai] < 0.0) s = -s;
    __syncwarp();
    for (int64_t i = lane; i < n; i += 32) x[i] *= s;
    if (lane == 0) {
        if (p.iters) p.iters[j] = conv ? its : -its;
        if (!conv) count_nonconverged(w, j);
    }
}

// Alg. 4 for the compact-WY cluster members: z_j = q / ||q||_2 with the first entry of
// largest magnitude made positive.  One warp per column, all columns in parallel.
__global__ void __launch_bounds__(kFirstWarps * 32) k_finalize(Problem p, Ws w)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kFirstWarps + warp;
    if (j >= p.M || w.head[j] == (int32_t)j) return;  // heads are final after k_first
    const JRef jr = jref(w, j);
    double* x = p.Z + jr.g->z + jr.jl * jr.g->ldz;
    const int64_t n = jr.g->n;
    if (!TINV_IN(p.zlen == 0 || dbg_range(jr.g->z + jr.jl * jr.g->ldz, jr.g->z + jr.jl * jr.g->ldz + n,
                                          p.zlen),
                 (int*)&w.ctr[kCtrErr]))
        return;
    double ss = 0.0, am = -1.0;
    int64_t ai = 0;
    for (int64_t i = lane; i < n; i += 32) {
        const double v = x[i];
        ss = fma(v, v, ss);
        if (fabs(v) > am) {
            am = fabs(v);
            ai = i;
        }
    }
    ss = warp_sum(ss);
    warp_argmax(am, ai);
    double sc = 1.0 / sqrt(ss);
    if (x[ai] < 0.0) sc = -sc;
    __syncwarp();
    for (int64_t i = lane; i < n; i += 32) x[i] *= sc;
}

// Solve for given right-hand sides (tinv_solve): one warp per column.
__global__ void __launch_bounds__(kFirstWarps * 32) k_solve_rhs(int64_t n, int64_t m, Ws w,
                                                                double* X, int64_t ldx, int scale)
{
    __shared__ double sh_all[kFirstWarps][8 * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kFirstWarps + warp;
    if (j >= m) return;
    double* x = X + j * ldx;
    if (scale) warp_scale(n, x, w.scal[0], w.u0n[j], lane);
    chunk_solve(n, fac_of(w, j, n), x, w.rhs + (size_t)j * (size_t)n, sh_all[warp], lane, 32,
                WarpSync());
}

// ==========================================================================================
// Persistent cluster kernel
// ==========================================================================================
// Phase profiling (separate diagnostic build with -DTINV_PHASE_PROFILE): thread 0 of each CTA
// accumulates clock64() per phase and prints the totals when the kernel ends.
#ifdef TINV_PHASE_PROFILE
enum { kPhLoad, kPhSolve, kPhA, kPhB1, kPhT1, kPhB2, kPhB, kPhB3, kPhT2, kPhB4, kPhC, kPhB5, kPhEnd,
       kPhT1a, kPhBa, kPhBb, kPhBc, kPhT2a, kPhT2b, kPhT2c, kPhCa, kPhCb, kPhN };
#define PROF_MARK(acc, i)                                   \
    do {                                                    \
        if (threadIdx.x == 0) {                             \
            long long _n = clock64();                       \
            (acc).c[i] += (unsigned long long)(_n - (acc).t); \
            (acc).t = _n;                                   \
        }                                                   \
    } while (0)
struct Prof {
    unsigned long long c[kPhN];
    long long t;
};
#else
#define PROF_MARK(acc, i) \
    do {                  \
    } while (0)
struct Prof {
    long long t;
};
#endif

struct Team {
    int32_t leader, G, rank;
    uint32_t* bar;
    uint32_t target;
};

struct ChainCtx {
    Problem p;
    Ws w;
    int32_t mode;
    const double* V;
    int64_t ldv;
    double* vsm;   // [n] working vector (shared or global)
    double* s1;    // [n] staging vector (shared or global)
    double* red;   // [2048] reduction / solve scratch (shared)
    double* xs;    // staging area of the blocked path (shared, Ws.xcap doubles) or null
    int* err;
    unsigned long long nsolve;  // solves so far (the team's stamps: equal in all its CTAs)
    Prof prof;
};

__device__ __forceinline__ int64_t part_lo(int64_t a, int64_t b, int r, int G)
{
    return a + ((b - a) * r) / G;
}

// Rows of passes A and C for rank r of G: the n rows of a lower trapezoid with K columns (row
// rho holds min(rho+1, K) of them).  For the one-member passes, while the triangle is a small
// part (4K <= n), equal rows are used (their short rows run less efficiently, so the smaller
// work does not make them cheaper); beyond that, ranges of equal work.  With c0 >= 0 (the
// multi-vector passes of the blocked path) always ranges of equal cost, a row costing
// min(rho+1, K) + c0.
__device__ __forceinline__ int64_t trap_row_lo(int64_t n, int64_t K, int r, int G, double c0 = -1.0)
{
    if (r <= 0) return 0;
    if (r >= G) return n;
    if (c0 < 0.0) {
        if (4 * K <= n) return (n * r) / G;
        c0 = 0.0;
    }
    const double Kd = (double)K, head = 0.5 * Kd * (Kd + 1.0) + c0 * Kd;
    const double total = head + (double)(n - K) * (Kd + c0);
    const double tgt = total * (double)r / (double)G;
    int64_t rho;
    if (tgt <= head) {
        const double b1 = 1.0 + 2.0 * c0;
        rho = (int64_t)llrint(0.5 * (sqrt(b1 * b1 + 8.0 * tgt) - b1));
    } else {
        rho = K + (int64_t)llrint((tgt - head) / (Kd + c0));
    }
    return min(n, max((int64_t)0, rho));
}

// Split [0, k) so that column i of an upper-triangular matrix (work i+1) is balanced.
__device__ __forceinline__ int64_t tri_col_lo(int64_t k, int r, int G)
{
    if (r <= 0) return 0;
    if (r >= G) return k;
    return min(k, (int64_t)llrint((double)k * sqrt((double)r / (double)G)));
}
// Split [0, k) so that row i of an upper-triangular matrix (work k-i) is balanced.
__device__ __forceinline__ int64_t tri_row_lo(int64_t k, int r, int G)
{
    if (r <= 0) return 0;
    if (r >= G) return k;
    return max((int64_t)0, k - (int64_t)llrint((double)k * sqrt(1.0 - (double)r / (double)G)));
}
// The same with a fixed cost of c0 columns per row (work k - i + c0): the rank with the short
// bottom rows gets fewer of them.  Cumulative work i (k + c0 + 1/2) - i^2 / 2 = its share.
__device__ __forceinline__ int64_t tri_row_lo_c(int64_t k, int r, int G, double c0)
{
    if (r <= 0) return 0;
    if (r >= G) return k;
    const double kd = (double)k, bq = 2.0 * kd + 2.0 * c0 + 1.0;
    const double tgt = (0.5 * kd * (kd + 1.0) + c0 * kd) * (double)r / (double)G;
    const double i = 0.5 * (bq - sqrt(fmax(0.0, bq * bq - 8.0 * tgt)));
    return min(k, max((int64_t)0, (int64_t)llrint(i)));
}

__device__ __forceinline__ int solve_group_size(int64_t n)
{
    int P = (int)ceil(sqrt(2.0 * (double)n));
    P = ((P + 31) / 32) * 32;
    return max(32, min(256, P));
}

// Sum (of v or of v^2) and max |v| (compared as bit patterns, no FP64 work) of cnt values in
// shared memory, reduced by 4 warps (one per SM sub-partition) and combined in a fixed order;
// every thread receives the results.  `red` holds >= 16 doubles.
template <bool SQUARE>
__device__ void cta_sum_max(const double* v, int64_t cnt, double* red, double& sum, double& mx)
{
    const int t = threadIdx.x, wid = t >> 5, lane = t & 31;
    unsigned long long* redu = (unsigned long long*)(red + 8);
    __syncthreads();
    if (wid < 4) {
        double a = 0.0;
        unsigned long long m = 0;
        for (int64_t i = wid * 32 + lane; i < cnt; i += 128) {
            const double x = v[i];
            a = SQUARE ? fma(x, x, a) : a + fabs(x);
            m = max(m, (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull);
        }
        a = warp_sum(a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            red[wid] = a;
            redu[wid] = m;
        }
    }
    __syncthreads();
    if (t == 0) {
        red[4] = (red[0] + red[1]) + (red[2] + red[3]);
        redu[4] = max(max(redu[0], redu[1]), max(redu[2], redu[3]));
    }
    __syncthreads();
    sum = red[4];
    mx = __longlong_as_double((long long)redu[4]);
    __syncthreads();
}

// Sum over the G ranks of a team of one partial (ranks `stride` doubles apart), in rank order,
// with the loads issued 8 at a time so the L2 latency is paid once per batch.
__device__ __forceinline__ double sum_partials(const double* base, size_t stride, int G)
{
    double acc = 0.0;
    int r = 0;
    for (; r + 8 <= G; r += 8) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldcg(base + (size_t)(r + q) * stride);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += v[q];
    }
    for (; r < G; ++r) acc += __ldcg(base + (size_t)r * stride);
    return acc;
}

// Warp-wide sum of slot `slot` of the per-rank scalar blocks of a team (lane-strided partial
// sums, then a fixed xor tree); called by a whole warp, every lane receives the result.
__device__ __forceinline__ double team_sum_slot(const double* scal_t, int G, int slot)
{
    const int lane = threadIdx.x & 31;
    double a = 0.0;
    for (int r = lane; r < G; r += 32) a += __ldcg(&scal_t[r * kScalTeam + slot]);
    return warp_sum(a);
}

// ---- compact-WY processing of one cluster by a team (Alg. 4, Sec. 3.3.2) -----------------
__device__ bool cwy_cluster(ChainCtx& cx, int32_t c, Team& tm)
{
    const Problem& p = cx.p;
    const Ws& w = cx.w;
    const int t = threadIdx.x;
    const int B = blockDim.x;
    const int G = tm.G, rank = tm.rank, leader = tm.leader;
    const int64_t s0 = w.clstart[c];
    const int64_t mc = w.clsize[c];
    const JRef jr = jref(w, s0);  // the cluster's problem; members are consecutive
    const Seg& sg = *jr.g;
    const int64_t n = sg.n;
    double* Zc = p.Z + sg.z + jr.jl * sg.ldz;  // column kk of Zc: member kk
    const int64_t ldz = sg.ldz;
    double* Tc = w.T + w.cltoff[c];
    const int64_t ldt = mc;
    double* Yc = w.Y + jr.off;  // Y column and factor rows of member kk at + kk n
    const size_t ns = (size_t)p.n;  // stride of the per-CTA buffers: the largest order
    double* vecS = w.vecS + (size_t)leader * ns;
    double* vecX = w.vecX + (size_t)leader * ns;
    double* vecR = w.vecR + (size_t)leader * ns;
    double* qbuf = w.qbuf + (size_t)leader * ns;
    double* vbuf = w.vbuf + (size_t)leader * ns;
    double* pubf = w.tpub + (size_t)leader * 8;  // 2 doubles per rank, then 6 per rank
    double* pubb = pubf + 2 * G;
    double* myS = w.partS + (size_t)(leader + rank) * ns;
    double* myG = w.partG + (size_t)(leader + rank) * ns;
    double* scal_t = w.partScal + (size_t)leader * kScalTeam;  // rank r at + r*kScalTeam
    double* vsm = cx.vsm;
    double* s1 = cx.s1;
    double* red = cx.red;
    const double onenrm = sg.onenrm, dtpcrt = sg.dtpcrt;
    const bool orth = (cx.mode == kModeOrth);
    __shared__ double s_b[8];
    // the cluster's ranges of Y, T, Z and of the team's buffers (TINV_DEBUG builds)
    if (!TINV_IN(s0 >= 0 && mc >= 1 && s0 + mc <= w.nM && n <= p.n && rank < G && leader + G <= w.P &&
                     dbg_range((int64_t)jr.off, (int64_t)jr.off + mc * n, w.nF) &&
                     dbg_range(w.cltoff[c], w.cltoff[c] + mc * mc, w.nTT) &&
                     dbg_range((int64_t)leader * p.n, (int64_t)(leader + G) * p.n, w.nPN) &&
                     (p.zlen == 0 || dbg_range(sg.z + jr.jl * ldz, sg.z + (jr.jl + mc - 1) * ldz + n, p.zlen)),
                 cx.err))
        return false;

    // rows of passes A and C and of the head step
    const int64_t ra0 = part_lo(0, n, rank, G), ra1 = part_lo(0, n, rank + 1, G);
    // Large teams add the team partials of s and g by slices (one CTA per slice, one more
    // barrier) instead of every CTA adding all G partials of every column it needs; the
    // additions are the same, in the same order, so the results do not change.
    const bool sliced = G >= kSliceTeam;

    int64_t kstart = 0;
    if (!orth) {
        // Alg. 4: Y_1 = [y_1], T_1 = [t_1] from the final head vector z.
        const double* z = Zc;
        double ss = 0.0;
        for (int64_t r = ra0 + t; r < ra1; r += B) ss = fma(z[r], z[r], ss);
        ss = block_sum(ss, red);
        if (t == 0) scal_t[rank * kScalTeam + 6] = ss;
        if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
        if (t < 32) {
            const double tot = team_sum_slot(scal_t, G, 6);
            const double nrm = sqrt(tot);
            const double z0 = z[0];
            const bool broke = !(nrm > 0.0) || !isfinite(nrm);
            const double cc = broke ? -1.0 : -sgn(z0) * nrm;
            const double u11 = broke ? 1.0 : z0;
            if (t == 0) {
                s_b[0] = cc;
                s_b[1] = 1.0 / (cc * cc - u11 * cc);
                s_b[2] = broke ? 1.0 : 0.0;
            }
        }
        __syncthreads();
        const double cc = s_b[0];
        const bool broke = s_b[2] != 0.0;
        for (int64_t r = ra0 + t; r < ra1; r += B) {
            double y = broke ? 0.0 : z[r];
            if (r == 0) y = broke ? 2.0 : z[0] - cc;
            Yc[r] = y;
        }
        if (rank == 0 && t == 0) Tc[0] = s_b[1];
        kstart = 1;
        // Y[:,0] and T[0,0] must be complete before members stage rows of Y
        if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
    }

    for (int64_t kk = kstart; kk < mc; ++kk) {
        const int64_t j = s0 + kk;
        const int64_t k = kk;  // previous reflectors: columns 0..k-1 of Yc
        // stage r = row k of Y_k into vecR (spread over the team)
        for (int64_t l = (int64_t)rank * B + t; l < k; l += (int64_t)G * B) vecR[l] = Yc[k + l * n];
        const Fac f = orth ? Fac{} : fac_at(w, jr.off + (size_t)kk * (size_t)n);
        const double u0n = orth ? 0.0 : w.u0n[j];
        // balanced bounds of this CTA's share of the T products (FP64 sqrt: one thread, once
        // per member; every CTA of the team computes the same values)
        __shared__ int64_t s_tb[6];
        if (t == 0) {
            s_tb[0] = tri_col_lo(k, rank, G);
            s_tb[1] = tri_col_lo(k, rank + 1, G);
            s_tb[2] = tri_row_lo(k, rank, G);
            s_tb[3] = tri_row_lo(k, rank + 1, G);
            // rows of passes A and C, balanced for the trapezoid of Y_{k+1}
            s_tb[4] = trap_row_lo(n, k + 1, rank, G);
            s_tb[5] = trap_row_lo(n, k + 1, rank + 1, G);
        }
        __syncthreads();
        const int64_t c0 = s_tb[0], c1 = s_tb[1], i0 = s_tb[2], i1 = s_tb[3];
        const int64_t rc0 = s_tb[4], rc1 = s_tb[5];
        // slices of the passes and T products: columns of Y_k / T_k and rows of Y
        if (!TINV_IN(dbg_range(c0, c1, k) && dbg_range(i0, i1, k) && dbg_range(rc0, rc1, n) &&
                         dbg_range(part_lo(k, n, rank, G), part_lo(k, n, rank + 1, G), n) && k < mc,
                     cx.err))
            return false;
        int nrmchk = 0, its = 0;
        bool conv = false;
        double fac_next = 0.0;
        const int maxits = orth ? 1 : kMaxIts;
        while (its < maxits) {
            ++its;
            // ---- the iterate v: rows [ra0, ra1) in shared memory, all rows in vsrc ----
            PROF_MARK(cx.prof, kPhEnd);
            const double* vsrc = orth ? cx.V + kk * cx.ldv : (its == 1 ? Zc + kk * ldz : vbuf);
            if (!orth && its > 1) {
                PROF_MARK(cx.prof, kPhLoad);
                // the solve of a sweep that cannot be the member's last only starts the next
                // sweep: a loose check suffices
                const bool may_end = nrmchk >= kExtra || its == maxits;
                TeamRef tr{tm.bar, &tm.target, G, rank, cx.err,
                           (unsigned long long*)(scal_t + 15), ++cx.nsolve,
                           (unsigned long long*)&w.ctr[kCtrFallback],
                           may_end ? kSolveTol : kSolveTolLoose, cx.p.spin_limit};
                if (!team_solve(n, f, qbuf, fac_next, vsm, vbuf, vecS, ra0, ra1, pubf, pubb, tr, red))
                    return false;
                PROF_MARK(cx.prof, kPhSolve);
            }
            // pass A's rows of v (all rows of vsrc are complete: the solve ends with a team
            // barrier, the first sweep's iterate was written before this kernel)
            if (orth || its == 1 || rc0 != ra0 || rc1 != ra1) {
                for (int64_t r = rc0 + t; r < rc1; r += B) vsm[r] = __ldcg(&vsrc[r]);
                __syncthreads();
            }
            PROF_MARK(cx.prof, kPhLoad);
            if (k > 0) {
                // ---- pass A: s = Y_k^T v = L_k^T v_check + Yhat_k^T v_hat (team partials) ----
                cta_coldots<kLower>(Yc, n, 0, k, rc0, rc1, vsm, red,
                                    [&](int64_t i, double s) { myS[i] = s; });
                PROF_MARK(cx.prof, kPhA);
                if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
                PROF_MARK(cx.prof, kPhB1);
                // ---- s' = T_k^T s, columns [c0, c1) of this CTA ----
                PROF_MARK(cx.prof, kPhB1);
                if (sliced) {
                    // each CTA adds the G partials of its slice of columns into vecX (free
                    // until the T column step); then every CTA reads the columns it needs
                    const int64_t l0 = part_lo(0, k, rank, G), l1 = part_lo(0, k, rank + 1, G);
                    for (int64_t l = l0 + t; l < l1; l += B)
                        vecX[l] = sum_partials(w.partS + (size_t)leader * ns + l, ns, G);
                    if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
                    for (int64_t l = t; l < c1; l += B) s1[l] = __ldcg(&vecX[l]);
                } else {
                    for (int64_t l = t; l < c1; l += B)
                        s1[l] = sum_partials(w.partS + (size_t)leader * ns + l, ns, G);
                }
                __syncthreads();
                PROF_MARK(cx.prof, kPhT1a);
                cta_coldots<kUpper>(Tc, ldt, c0, c1, 0, k, s1, red,
                                    [&](int64_t i, double s) { vecS[i] = s; });
                PROF_MARK(cx.prof, kPhT1);
                if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
                PROF_MARK(cx.prof, kPhB2);
                for (int64_t l = t; l < k; l += B) s1[l] = __ldcg(&vecS[l]);
                __syncthreads();
            }
            // ---- pass B: u_hat = v_hat - Yhat_k s' (rows [k, n) split over the team) ----
            const int64_t rb0 = part_lo(k, n, rank, G), rb1 = part_lo(k, n, rank + 1, G);
            for (int64_t r = rb0 + t; r < rb1; r += B) vsm[r] = __ldcg(&vsrc[r]);
            __syncthreads();
            PROF_MARK(cx.prof, kPhBa);
            if (k > 0) {
                cta_rowdots<kAllCols, 1>(Yc, n, rb0, rb1, k, s1, nullptr, red,
                                         [&](int64_t rho, double a, double) { vsm[rho] -= a; });
            }
            PROF_MARK(cx.prof, kPhBb);
            double uu, umx;
            cta_sum_max<true>(vsm + rb0, rb1 - rb0, red, uu, umx);
            PROF_MARK(cx.prof, kPhBc);
            if (k > 0) {
                // g_u = Yhat_k^T u_hat (partial over this CTA's rows)
                cta_coldots<kLower>(Yc, n, 0, k, rb0, rb1, vsm, red,
                                    [&](int64_t i, double s) { myG[i] = s; });
            }
            if (t == 0) {
                scal_t[rank * kScalTeam + 0] = uu;
                scal_t[rank * kScalTeam + 1] = (rb0 <= k && k < rb1) ? vsm[k] : 0.0;
            }
            PROF_MARK(cx.prof, kPhB);
            if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhB3);
            // ---- g = Yhat_k^T u_hat from the team partials (all warps but the first), while
            //      warp 0 forms the reflector (Eq. yt with t = 1/(c^2 - u_kk c), Sec. 3.3.2) ----
            if (t < 32) {
                double tot = 0.0, ukk = 0.0;
                for (int r = t; r < G; r += 32) {
                    tot += __ldcg(&scal_t[r * kScalTeam + 0]);
                    ukk += __ldcg(&scal_t[r * kScalTeam + 1]);
                }
                tot = warp_sum(tot);
                ukk = warp_sum(ukk);
                const double nrm = sqrt(tot);
                const bool broke = !(nrm > 0.0) || !isfinite(nrm);
                const double cc = broke ? -1.0 : -sgn(ukk) * nrm;
                const double ue = broke ? 1.0 : ukk;
                if (t == 0) {
                    s_b[0] = cc;
                    s_b[1] = 1.0 / (cc * cc - ue * cc);  // t_k
                    s_b[2] = ue - cc;                    // y_kk
                    s_b[3] = broke ? 1.0 : 0.0;
                }
            } else if (sliced) {
                // the slice of g of this CTA into vecS (free after pass B)
                const int64_t l0 = part_lo(0, k, rank, G), l1 = part_lo(0, k, rank + 1, G);
                for (int64_t l = l0 + (t - 32); l < l1; l += B - 32)
                    vecS[l] = sum_partials(w.partG + (size_t)leader * ns + l, ns, G);
            } else {
                for (int64_t l = i0 + (t - 32); l < k; l += B - 32)
                    s1[l] = sum_partials(w.partG + (size_t)leader * ns + l, ns, G);
            }
            if (sliced) {
                if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
                for (int64_t l = i0 + t; l < k; l += B) s1[l] = __ldcg(&vecS[l]);
            }
            __syncthreads();
            const double cc = s_b[0], tk = s_b[1], ykk = s_b[2];
            const bool broke = s_b[3] != 0.0;
            PROF_MARK(cx.prof, kPhT2a);
            // ---- T column: t_hat = -t_k T_k (Yhat_k^T y_hat) with Yhat^T y_hat = g_u - c r;
            //      and x_T = T_{k+1} (row k of Y_{k+1}) = [T_k r + t_hat y_kk ; t_k y_kk] ----
            if (broke) {  // u_hat := e_1, so g_u = Yhat^T e_1 = r
                for (int64_t l = i0 + t; l < k; l += B) s1[l] = __ldcg(&vecR[l]);
                __syncthreads();
            }
            // second vector (r) read through a shared copy of vecR
            double* rsm = (double*)vecR;  // read-only from here on
            cta_rowdots<kUpperCol, 2>(Tc, ldt, i0, i1, k, s1, rsm, red,
                                      [&](int64_t i, double a, double b) {
                                          const double th = -tk * fma(-cc, b, a);
                                          Tc[i + kk * ldt] = th;
                                          vecX[i] = fma(th, ykk, b);
                                      });
            PROF_MARK(cx.prof, kPhT2c);
            if (rank == 0 && t == 0) {
                Tc[kk + kk * ldt] = tk;
                vecX[kk] = tk * ykk;
            }
            // Y column k: rows of pass B (u_hat, with the diagonal entry u_kk - c)
            for (int64_t r = rb0 + t; r < rb1; r += B) {
                double y = broke ? 0.0 : vsm[r];
                if (r == k) y = ykk;
                Yc[r + kk * n] = y;
            }
            PROF_MARK(cx.prof, kPhT2);
            if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhB4);
            // ---- pass C: q = (Y_{k+1} T_{k+1} Y_{k+1}^T - I) e_k = Y_{k+1} x_T - e_k ----
            for (int64_t l = t; l <= k; l += B) s1[l] = __ldcg(&vecX[l]);
            __syncthreads();
            PROF_MARK(cx.prof, kPhCa);
            cta_rowdots<kLowerCol, 1>(Yc, n, rc0, rc1, k + 1, s1, nullptr, red,
                                      [&](int64_t rho, double a, double) {
                                          const double q = (rho == k) ? a - 1.0 : a;
                                          qbuf[rho] = q;
                                          vsm[rho] = q;
                                      });
            // per sweep only sum|q| (the next scaling) and max|q| (the test) are needed; the
            // 2-norm and the sign convention are applied once, by k_finalize
            PROF_MARK(cx.prof, kPhCb);
            double as, am;
            cta_sum_max<false>(vsm + rc0, rc1 - rc0, red, as, am);
            if (t == 0) {
                scal_t[rank * kScalTeam + 2] = as;
                scal_t[rank * kScalTeam + 3] = am;
            }
            PROF_MARK(cx.prof, kPhC);
            if (!team_sync(tm.bar, tm.target, G, cx.err, cx.p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhB5);
            if (orth) {
                for (int64_t r = ra0 + t; r < ra1; r += B)
                    Zc[r + kk * ldz] = qbuf[r];
                break;
            }
            // ---- team statistics, convergence test on x = -c q (||x||_inf = |c| max|q|) ----
            if (t < 32) {
                const double A1 = team_sum_slot(scal_t, G, 2);
                unsigned long long mb = 0;
                for (int r = t; r < G; r += 32)
                    mb = max(mb, (unsigned long long)__double_as_longlong(__ldcg(&scal_t[r * kScalTeam + 3])));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
                if (t == 0) {
                    s_b[4] = A1;
                    s_b[5] = __longlong_as_double((long long)mb);
                }
            }
            __syncthreads();
            const double A1 = s_b[4], M = s_b[5];
            const bool success = !broke && fabs(cc) * M >= dtpcrt;
            if (success && ++nrmchk >= kExtra + 1) conv = true;
            if (conv || its == maxits) {
                // Alg. 4 (normalization and sign) is applied by k_finalize
                for (int64_t r = ra0 + t; r < ra1; r += B) Zc[r + kk * ldz] = qbuf[r];
                if (rank == 0 && t == 0) {
                    if (p.iters) p.iters[j] = conv ? its : -its;
                    if (!conv) count_nonconverged(w, j);
                }
                break;
            }
            // next sweep's scaled input: scl * x = q * (-sgn(c) n ||T||_1 max(eps,|u_nn|) / sum|q|)
            if (t == 0) s_b[6] = -sgn(cc) * (((double)n * onenrm) * fmax(kEps, u0n)) / A1;
            __syncthreads();
            fac_next = s_b[6];
        }
    }
    return true;
}

#include "tinv_block.cuh"

// ---- MGS processing of one cluster by one CTA (Alg. 1) -----------------------------------
__device__ bool mgs_cluster(ChainCtx& cx, int32_t c)
{
    const Problem& p = cx.p;
    const Ws& w = cx.w;
    const int t = threadIdx.x, B = blockDim.x;
    const int64_t s0 = w.clstart[c];
    const int64_t mc = w.clsize[c];
    const JRef jr = jref(w, s0);  // the cluster's problem; members are consecutive
    const Seg& sg = *jr.g;
    const int64_t n = sg.n;
    double* Zc = p.Z + sg.z + jr.jl * sg.ldz;  // column kk of Zc: member kk
    const int64_t ldz = sg.ldz;
    double* v = cx.vsm;
    double* red = cx.red;
    const bool orth = (cx.mode == kModeOrth);
    const double onenrm = sg.onenrm, dtpcrt = sg.dtpcrt;
    const int64_t kstart = orth ? 0 : 1;
    if (!TINV_IN(s0 >= 0 && mc >= 1 && s0 + mc <= w.nM && n <= p.n &&
                     (orth || dbg_range((int64_t)jr.off, (int64_t)jr.off + mc * n, w.nF)) &&
                     (p.zlen == 0 || dbg_range(sg.z + jr.jl * ldz, sg.z + (jr.jl + mc - 1) * ldz + n, p.zlen)),
                 cx.err))
        return false;
    for (int64_t kk = kstart; kk < mc; ++kk) {
        const int64_t j = s0 + kk;
        const Fac f = orth ? Fac{} : fac_at(w, jr.off + (size_t)kk * (size_t)n);
        const double u0n = orth ? 0.0 : w.u0n[j];
        int nrmchk = 0, its = 0, attempt = 0;
        bool conv = false;
        const int maxits = orth ? 1 : kMaxIts;
        while (its < maxits) {
            ++its;
            if (orth) {
                for (int64_t r = t; r < n; r += B) v[r] = cx.V[r + kk * cx.ldv];
                __syncthreads();
            } else if (its == 1) {
                for (int64_t r = t; r < n; r += B) v[r] = Zc[r + kk * ldz];
                __syncthreads();
            } else {
                double as = 0.0;
                for (int64_t r = t; r < n; r += B) as += fabs(v[r]);
                as = block_sum(as, red);
                __shared__ double s_scl;
                if (t == 0) s_scl = ((double)n * onenrm) * fmax(kEps, u0n) / as;
                __syncthreads();
                const double scl = s_scl;
                uint32_t tgt = 0;
                const bool may_end = nrmchk >= kExtra || its == maxits;
                TeamRef tr{nullptr, &tgt, 1, 0, cx.err, nullptr, 0ull,
                           (unsigned long long*)&w.ctr[kCtrFallback],
                           may_end ? kSolveTol : kSolveTolLoose, 0u};
                if (!team_solve(n, f, v, scl, v, nullptr, cx.s1, 0, n, nullptr, nullptr, tr, red))
                    return false;
            }
            // Alg. 1: v <- v - <v, z_i> z_i for the previous members, in order
            for (int64_t i = 0; i < kk; ++i) {
                const double* zi = Zc + i * ldz;
                double h = 0.0;
                for (int64_t r = t; r < n; r += B) h = fma(v[r], zi[r], h);
                h = block_sum(h, red);
                for (int64_t r = t; r < n; r += B) v[r] = fma(-h, zi[r], v[r]);
                __syncthreads();
            }
            double as = 0.0, mx = 0.0;
            for (int64_t r = t; r < n; r += B) {
                as += fabs(v[r]);
                mx = fmax(mx, fabs(v[r]));
            }
            as = block_sum(as, red);
            mx = block_max(mx, red);
            bool ok = true;
            if (!(as > 0.0) && !orth) {
                // breakdown: restart from a fresh random vector
                ++attempt;
                const uint64_t key = start_key(sg.seed, sg.kj0 + jr.jl + kk, attempt);
                for (int64_t r = t; r < n; r += B) v[r] = start_value(key, r);
                __syncthreads();
                ok = false;
            }
            if (orth) break;
            if (ok && mx >= dtpcrt && ++nrmchk >= kExtra + 1) {
                conv = true;
                break;
            }
        }
        // normalize; first entry of largest magnitude positive (orth: unit vector only)
        double ss = 0.0, am = -1.0;
        int64_t ai = n;
        for (int64_t r = t; r < n; r += B) {
            ss = fma(v[r], v[r], ss);
            if (fabs(v[r]) > am) {
                am = fabs(v[r]);
                ai = r;
            }
        }
        ss = block_sum(ss, red);
        {
            warp_argmax(am, ai);
            __shared__ double s_am[32];
            __shared__ int64_t s_ai[32];
            const int lane = t & 31, wid = t >> 5;
            if (lane == 0) {
                s_am[wid] = am;
                s_ai[wid] = ai;
            }
            __syncthreads();
            if (wid == 0) {
                double a3 = lane < (B >> 5) ? s_am[lane] : -1.0;
                int64_t i3 = lane < (B >> 5) ? s_ai[lane] : n;
                warp_argmax(a3, i3);
                if (lane == 0) s_ai[0] = i3;
            }
            __syncthreads();
            ai = (s_ai[0] >= 0 && s_ai[0] < n) ? s_ai[0] : 0;
        }
        double sc = 1.0 / sqrt(ss);
        if (!orth && v[ai] < 0.0) sc = -sc;
        double* dst = Zc + kk * ldz;
        for (int64_t r = t; r < n; r += B) dst[r] = v[r] * sc;
        __syncthreads();
        if (!orth && t == 0) {
            if (p.iters) p.iters[j] = conv ? its : -its;
            if (!conv) count_nonconverged(w, j);
        }
        if (ld_volatile_i32(cx.err) != 0) return false;
    }
    return true;
}

// METHOD 0: compact WY, one member at a time; 1: MGS; 2: compact WY with blocks of members on
// CTA teams (tinv_opts.block), one member at a time elsewhere.
template <int METHOD, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_chain(Problem p, Ws w, int32_t mode,
                                                           const double* V, int64_t ldv)
{
    extern __shared__ double smem[];
    const int b = blockIdx.x, t = threadIdx.x;
    const int64_t n = p.n;
    ChainCtx cx;
    cx.p = p;
    cx.w = w;
    cx.mode = mode;
    cx.V = V;
    cx.ldv = ldv;
    cx.red = smem;  // 2048 doubles
    cx.xs = nullptr;
    if (w.use_smem) {
        cx.vsm = smem + 2048;
        cx.s1 = smem + 2048 + n;
        if (w.block >= 2 && w.xcap > 0) cx.xs = smem + 2048 + 2 * n + 64;  // 64: panel slack
    } else {
        cx.vsm = w.gvec + (size_t)b * 2 * (size_t)n;
        cx.s1 = cx.vsm + n;
    }
    cx.err = (int*)&w.ctr[kCtrErr];
    cx.nsolve = 0;
    __shared__ int s_c;
#ifdef TINV_PHASE_PROFILE
    for (int i = 0; i < kPhN; ++i) cx.prof.c[i] = 0;
    const long long t_begin = clock64();
#endif
    cx.prof.t = clock64();

    const int32_t tf = w.sched[4 * b + 0], tg = w.sched[4 * b + 1], tr = w.sched[4 * b + 2],
                  tc = w.sched[4 * b + 3];
    if (!TINV_IN(tf >= 0 && tg >= 1 && tf + tg <= w.P && tr >= 0 && tr < tg && tc < (int32_t)w.nM,
                 (int*)&w.ctr[kCtrErr]))
        return;
    if (tc >= 0) {
        Team tm{tf, tg, tr, w.bar + tf, 0u};
        bool ok;
        if (METHOD == 2) {  // compact WY with blocks of members where the team's cluster allows
            const int nbk = cx.xs ? block_members(w, w.clsize[tc], tg, w.segs[w.segj[w.clstart[tc]]].n) : 1;
            ok = (nbk >= 2) ? bcwy_cluster(cx, tc, tm, nbk) : cwy_cluster(cx, tc, tm);
        } else if (METHOD == 0) {
            ok = cwy_cluster(cx, tc, tm);
        } else {
            ok = mgs_cluster(cx, tc);
        }
        if (!ok) return;
    }
    const int64_t nq = w.ctr[kCtrNQueue];
    for (;;) {
        if (t == 0) {
            const unsigned long long q =
                atomicAdd((unsigned long long*)&w.ctr[kCtrQHead], 1ull);
            s_c = ((int64_t)q < nq && ld_volatile_i32(cx.err) == 0) ? w.queue[q] : -1;
        }
        __syncthreads();
        const int32_t c = s_c;
        __syncthreads();
        if (c < 0) break;
        if (!TINV_IN(c < (int32_t)w.nM, cx.err)) return;
        Team tm{b, 1, 0, w.bar + b, 0u};
        bool ok;
        if (METHOD == 2) {  // the blocked form also on a CTA alone where the cluster allows
            const int nbk = cx.xs ? block_members(w, w.clsize[c], 1, w.segs[w.segj[w.clstart[c]]].n) : 1;
            ok = (nbk >= 2) ? bcwy_cluster(cx, c, tm, nbk) : cwy_cluster(cx, c, tm);
        } else {
            ok = (METHOD != 1) ? cwy_cluster(cx, c, tm) : mgs_cluster(cx, c);
        }
        if (!ok) return;
    }
#ifdef TINV_PHASE_PROFILE
    if (t == 0) {
        const unsigned long long* sp = g_solve_prof + (size_t)b * kSolvePh;
        printf("SPROF cta=%d team=%d G=%d sv_stage=%llu sv_fwd1=%llu sv_fcarry=%llu sv_fwd2=%llu sv_back1=%llu "
               "sv_bfold=%llu sv_back2=%llu sv_check=%llu\n",
               b, tc, tg, sp[0], sp[1], sp[2], sp[3], sp[4], sp[5], sp[6], sp[7]);
    }
    if (t == 0)
        printf("PROF cta=%d team=%d G=%d total=%lld load=%llu solve=%llu A=%llu b1=%llu T1red=%llu T1=%llu "
               "b2=%llu Bload=%llu Brow=%llu Bsum=%llu B=%llu b3=%llu T2refl=%llu T2red=%llu T2row=%llu "
               "T2=%llu b4=%llu Cload=%llu Crow=%llu C=%llu b5=%llu end=%llu\n",
               b, tc, tg, clock64() - t_begin, cx.prof.c[kPhLoad], cx.prof.c[kPhSolve], cx.prof.c[kPhA],
               cx.prof.c[kPhB1], cx.prof.c[kPhT1a], cx.prof.c[kPhT1], cx.prof.c[kPhB2], cx.prof.c[kPhBa],
               cx.prof.c[kPhBb], cx.prof.c[kPhBc], cx.prof.c[kPhB], cx.prof.c[kPhB3], cx.prof.c[kPhT2a],
               cx.prof.c[kPhT2b], cx.prof.c[kPhT2c], cx.prof.c[kPhT2], cx.prof.c[kPhB4], cx.prof.c[kPhCa],
               cx.prof.c[kPhCb], cx.prof.c[kPhC], cx.prof.c[kPhB5], cx.prof.c[kPhEnd]);
#endif
}

// ==========================================================================================
// Launchers
// ==========================================================================================
// Threads per CTA of the cluster kernel (one CTA per SM).  Two 256-thread CTAs per SM measured
// slower on the glued-Wilkinson workload (173.2 against 170.6 ms) and on the 512-problem batch
// (205k against 224k eigenvectors/s): the CTAs sharing an SM belong to teams that run the same
// phases at the same time.
int32_t chain_threads(int64_t)
{
    return 512;
}

bool chain_use_smem(int64_t n)
{
    return (size_t)(2048 + 2 * n) * sizeof(double) + 4096 <= 220u * 1024u;
}

size_t chain_smem_bytes(int64_t n, bool use_smem, int32_t xcap)
{
    return (size_t)(2048 + (use_smem ? 2 * n : 0) + (use_smem && xcap > 0 ? xcap + 64 : 0)) * sizeof(double);
}

int32_t block_xcap(int64_t n)
{
    if (!chain_use_smem(n)) return 0;
    // 227 KB of shared memory per CTA, 8 KB of it left for the kernel's static arrays.  The area
    // holds the CTA-local solves' scratch and the staged vectors of small blocks only: larger
    // blocks read theirs from the team's buffers in L2, which measured faster than a larger area
    // (every KB of it is taken from the L1 that the passes' reads of Y go through; glued
    // n = 4200: 89.8 ms with 4 K doubles, 92.4 ms with 16 K)
    const int64_t avail = (int64_t)(227 * 1024 - 8 * 1024) / 8 - 2048 - 2 * n - 64 - 512;
    return (int32_t)max((int64_t)0, min((int64_t)4096, avail));
}

int32_t chain_grid(int32_t cap, int64_t)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int32_t P = sms > 0 ? sms : 1;
    if (cap > 0 && cap < P) P = cap;
    return P;
}

cudaError_t launch_plan(const Problem& p, const Ws& w, int32_t max_team, cudaStream_t st)
{
    if (p.nseg <= 0) return cudaSuccess;
    k_plan_seg<<<(unsigned)p.nseg, kPlanThreads, 0, st>>>(p, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_plan_list<<<1, kPlanThreads, 0, st>>>(p, w, max_team);
    return cudaGetLastError();
}

cudaError_t launch_norm(const Problem& p, const Ws& w, cudaStream_t st)
{
    k_norm<<<1, kPlanThreads, 0, st>>>(p, w);
    return cudaGetLastError();
}

cudaError_t launch_orth_plan(const Problem& p, const Ws& w, int32_t method, cudaStream_t st)
{
    k_orth_plan<<<1, 256, 0, st>>>(p, w, method);
    return cudaGetLastError();
}

cudaError_t launch_lu(int64_t n, const double* d, const double* e, int64_t m, const double* shift,
                      double* l, double* u0_or_r, double* u1, double* u2, uint8_t* piv,
                      double* u0n, double* tolv, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    const int th = 32;  // one warp per block spreads the sequential factorizations over SMs
    const unsigned blocks = (unsigned)((m + th - 1) / th);
    k_lu<<<blocks, th, 0, st>>>(n, d, e, m, shift, l, u0_or_r, u1, u2, piv, u0n, tolv);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || !tolv) return err;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned rb = (unsigned)min(m, (int64_t)(sms > 0 ? sms : 1) * 8);
    k_recip<<<rb, 256, 0, st>>>(n, m, u0_or_r, u1, u2, tolv);
    return cudaGetLastError();
}

static int device_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

cudaError_t launch_lu_seg(const Problem& p, const Ws& w, cudaStream_t st)
{
    if (p.M <= 0) return cudaSuccess;
    // one warp per block spreads the sequential factorizations over the SMs; with fewer than
    // 32 shifts per SM each warp takes ceil(M / SMs) shifts, so that every SM gets one
    const int sms = device_sms();
    const int64_t per = (p.M + sms - 1) / sms;
    const int lanes = (int)(per < 32 ? per : 32);
    k_lu_seg<<<(unsigned)((p.M + lanes - 1) / lanes), 32, 0, st>>>(p, w, lanes);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const unsigned rb = (unsigned)min(p.M, (int64_t)sms * 8);
    k_recip_seg<<<rb, 256, 0, st>>>(p, w);
    return cudaGetLastError();
}

cudaError_t launch_first(const Problem& p, const Ws& w, cudaStream_t st)
{
    if (p.M <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((p.M + kFirstWarps - 1) / kFirstWarps);
    k_first<<<blocks, kFirstWarps * 32, 0, st>>>(p, w);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Problem& p, const Ws& w, cudaStream_t st)
{
    if (p.M <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((p.M + kFirstWarps - 1) / kFirstWarps);
    k_finalize<<<blocks, kFirstWarps * 32, 0, st>>>(p, w);
    return cudaGetLastError();
}

cudaError_t launch_solve_rhs(int64_t n, int64_t m, const Ws& w, double* X, int64_t ldx,
                             int32_t scale, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((m + kFirstWarps - 1) / kFirstWarps);
    k_solve_rhs<<<blocks, kFirstWarps * 32, 0, st>>>(n, m, w, X, ldx, scale);
    return cudaGetLastError();
}

cudaError_t launch_chain(const Problem& p, const Ws& w, int32_t mode, const double* V, int64_t ldv,
                         cudaStream_t st)
{
    const size_t smem = chain_smem_bytes(p.n, w.use_smem != 0, w.block >= 2 ? w.xcap : 0);
    const int nt = chain_threads(p.n);
    void* fn;
    if (p.method == 0)
        fn = (w.block >= 2 && w.xcap > 0) ? (void*)k_chain<2, 512> : (void*)k_chain<0, 512>;
    else
        fn = (void*)k_chain<1, 512>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, occ = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1 || (int64_t)occ * sms < w.P) return cudaErrorCooperativeLaunchTooLarge;
    Problem pp = p;
    Ws ww = w;
    int32_t mm = mode;
    const double* VV = V;
    int64_t ll = ldv;
    void* args[] = {&pp, &ww, &mm, &VV, &ll};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)w.P), dim3((unsigned)nt), args, smem, st);
}

}  // namespace tinvx
