// tinv_block.cuh -- blocked compact-WY reorthogonalization of a cluster by a CTA team
// (tinv_opts.block >= 2): the members after the cluster's head are split into blocks of at most
// nb that sweep together, block b holding the members 1 + b + nblk c (nblk blocks): the members
// of a block are spread evenly over the cluster, and near neighbours in the spectrum, in
// different blocks, are orthogonalized against finished vectors.  Per block sweep, each member's
// iterate is solved on its own CTA of the team (no team barrier inside a solve), then the whole
// block is orthogonalized by the compact-WY block form of Sec. 3.2 (Eqs. cwy1/cwy2):
// W = (I - Y T^T Y^T) V with one pass over Y for all bb iterates, a Householder QR of the
// block's panel (one team barrier per column), T extended by Eq. cwy1 with triangular products
// over T for all columns, and the bb vectors q = (Y T Y^T - I) e_col with one more pass over Y.
// The vectors the passes and products share (the team's sums of S, S', the Gram rows, X_T) are
// staged in shared memory for small blocks and read from the team's buffers in L2 otherwise.
// A sweep takes bb + 6 team barriers (bb + 8 where the team sums S and the Gram rows once by
// slices), where one member at a time takes about 9 per member.  Included by tinv_kernels.cu
// inside its namespace (it uses the cluster kernel's context and the helpers defined there).
#pragma once

// Row-major staged vectors in shared memory: x_c[idx] = p[idx * ld + c].
struct XRow {
    const double* p;
    int ld;
    __device__ __forceinline__ double operator()(int64_t idx, int c) const { return p[idx * ld + c]; }
};
// Column vectors in shared memory holding rows [off, off + ld): x_c[idx] = p[c * ld + idx - off].
struct XCol {
    const double* p;
    int64_t ld, off;
    __device__ __forceinline__ double operator()(int64_t idx, int c) const { return p[c * ld + idx - off]; }
};
// Row-major vectors in global memory written by other CTAs (read through L2): p[idx * ld + c].
struct XGRow {
    const double* p;
    int64_t ld;
    __device__ __forceinline__ double operator()(int64_t idx, int c) const { return __ldcg(p + idx * ld + c); }
};
// Column vectors in global memory written by other CTAs (read through L2): base + c * ld + idx.
struct XGlob {
    const double* base;
    int64_t ld;
    __device__ __forceinline__ double operator()(int64_t idx, int c) const { return __ldcg(base + c * ld + idx); }
};

// Multi-vector column products: out(i, c, sum_{r in R(i)} A[r + i lda] x_c[r]) for columns i in
// [c0, c1) and vectors c < nv (nv <= NV), R(i) as cta_coldots (LOWER: [max(rlo, i), rhi),
// UPPER: [rlo, min(rhi, i + 1))).  A warp takes 32/RP columns x RP row phases; every load of A
// feeds nv FMAs (8 columns x 4 phases measured faster than 4 x 8: glued n = 4200 90.0 against
// 92.0 ms, Toeplitz n = 4200 1.26 against 1.57 s).  Rows are split into segments when the columns alone do not fill the warps; the
// segment partials are added by a fixed-shape tree, so results do not depend on scheduling.
template <int KIND, int NV, class XF, class Out, int RP = 4>
__device__ __noinline__ void mv_coldots(const double* __restrict__ A, int64_t lda, int64_t c0, int64_t c1,
                                        int64_t rlo, int64_t rhi, XF xf, int nv, double* red, Out out)
{
    constexpr int CW = 32 / RP;  // columns per warp
    const int nW = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl = lane / RP, ph = lane % RP;
    const int64_t nc = c1 - c0;
    if (nc <= 0 || nv <= 0) return;
    if (KIND == kLower)
        rlo = max(rlo, c0);
    else
        rhi = min(rhi, c1);
    const int64_t groups = (nc + CW - 1) / CW;
    const int64_t rows = rhi > rlo ? rhi - rlo : 0;
    int lmax = 0;
    while (lmax < 4 && ((int64_t)nc * nv << (lmax + 1)) <= 2048 && rows >= ((int64_t)8 * RP << (lmax + 1))) ++lmax;
    const int lS = pick_segments(groups, (rows + RP - 1) / RP * nv, nW, lmax);
    const int S = 1 << lS;
    const int64_t seglen = (rows + S - 1) >> lS;
    const int64_t units = groups << lS;
    for (int64_t u = wid; u < units; u += nW) {
        const int64_t g = u >> lS;
        const int sg = (int)(u & (S - 1));
        const int64_t i = c0 + g * CW + cl;
        const bool act = i < c1;
        const int64_t s_lo = rlo + sg * seglen, s_hi = min(rhi, s_lo + seglen);
        int64_t a = 0, b = 0;
        if (act) {
            a = max(s_lo, (KIND == kLower) ? max(rlo, i) : rlo);
            b = min(s_hi, (KIND == kLower) ? rhi : min(rhi, i + 1));
        }
        double acc[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = 0.0;
        if (act && a < b) {
            const double* col = A + i * lda;
            int64_t r = a + ((ph - a) & (RP - 1));
            for (; r + RP < b; r += 2 * RP) {
                const double y0 = col[r], y1 = col[r + RP];
#pragma unroll
                for (int c = 0; c < NV; ++c)
                    if (c < nv) acc[c] = fma(y1, xf(r + RP, c), fma(y0, xf(r, c), acc[c]));
            }
            if (r < b) {
                const double y0 = col[r];
#pragma unroll
                for (int c = 0; c < NV; ++c)
                    if (c < nv) acc[c] = fma(y0, xf(r, c), acc[c]);
            }
        }
#pragma unroll
        for (int o = 1; o < RP; o <<= 1) {
#pragma unroll
            for (int c = 0; c < NV; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        }
        if (act && ph == 0) {
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                if (c >= nv) break;
                if (S == 1)
                    out(i, c, acc[c]);
                else
                    red[((int64_t)sg * nc + (i - c0)) * nv + c] = acc[c];
            }
        }
    }
    if (S > 1) {
        tree_segments(red, S, nc, nv);
        for (int64_t q = threadIdx.x; q < nc * nv; q += blockDim.x) out(c0 + q / nv, (int)(q % nv), red[q]);
    }
    __syncthreads();
}

// Multi-vector row products: out(rho, c, sum_{i in C(rho)} A[rho + i lda] x_c[i]) for rows rho in
// [r0, r1) and vectors c < nv, C(rho) as cta_rowdots (LOWERCOL: [0, min(ccap, rho + 1)),
// UPPERCOL: [rho, ccap), ALL: [0, ccap)).  A warp takes RL consecutive rows x 32/RL column
// phases; column ranges are split into segments when the rows alone do not fill the warps.
// The lanes of a row group step through the same columns (for UPPERCOL from the group's first
// row, the entries left of a lane's own row masked), so that each load of A is RL consecutive
// doubles of one column and each x_c[i] one broadcast value.
template <int RL, int KIND, int NV, class XF, class Out>
__device__ __noinline__ void mv_rowdots_rl(const double* __restrict__ A, int64_t lda, int64_t r0, int64_t r1,
                                           int64_t ccap, XF xf, int nv, double* red, Out out)
{
    constexpr int CL = 32 / RL;
    const int nW = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rr = lane % RL, ph = lane / RL;
    const int64_t nr = r1 - r0;
    const int64_t rgroups = (nr + RL - 1) / RL;
    const int64_t gb = (KIND == kUpperCol) ? r0 : 0;
    const int64_t ge = (KIND == kLowerCol) ? min(ccap, r1) : ccap;
    const int64_t glen = ge > gb ? ge - gb : 0;
    int lmax = 0;
    while (lmax < 5 && ((int64_t)nr * nv << (lmax + 1)) <= 2048 && glen >= ((int64_t)8 * CL << (lmax + 1))) ++lmax;
    const int lS = pick_segments(rgroups, (glen + CL - 1) / CL * nv, nW, lmax);
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
            const int64_t cb = (KIND == kUpperCol) ? r0 + g * RL : 0;  // the group's first row
            const int64_t ce = (KIND == kLowerCol) ? min(ccap, rho + 1) : ccap;
            a = max(s0, cb);
            b = min(s1, ce);
        }
        double acc[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = 0.0;
        if (act && a < b) {
            const double* row = A + rho;
            // UPPERCOL: columns i < rho of this lane's row are not its terms (masked to 0)
            auto ld = [&](int64_t i) { return (KIND != kUpperCol || i >= rho) ? row[i * lda] : 0.0; };
            int64_t i = a + (((int64_t)ph - a) % CL + CL) % CL;
            for (; i + CL < b; i += 2 * CL) {
                const double y0 = ld(i), y1 = ld(i + CL);
#pragma unroll
                for (int c = 0; c < NV; ++c)
                    if (c < nv) acc[c] = fma(y1, xf(i + CL, c), fma(y0, xf(i, c), acc[c]));
            }
            if (i < b) {
                const double y0 = ld(i);
#pragma unroll
                for (int c = 0; c < NV; ++c)
                    if (c < nv) acc[c] = fma(y0, xf(i, c), acc[c]);
            }
        }
#pragma unroll
        for (int o = RL; o < 32; o <<= 1) {
#pragma unroll
            for (int c = 0; c < NV; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        }
        if (act && ph == 0) {
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                if (c >= nv) break;
                if (S == 1)
                    out(rho, c, acc[c]);
                else
                    red[((int64_t)sg * nr + (rho - r0)) * nv + c] = acc[c];
            }
        }
    }
    if (S > 1) {
        tree_segments(red, S, nr, nv);
        for (int64_t q = threadIdx.x; q < nr * nv; q += blockDim.x) out(r0 + q / nv, (int)(q % nv), red[q]);
    }
    __syncthreads();
}

template <int KIND, int NV, class XF, class Out>
__device__ __forceinline__ void mv_rowdots_nv(const double* __restrict__ A, int64_t lda, int64_t r0, int64_t r1,
                                              int64_t ccap, XF xf, int nv, double* red, Out out)
{
    // groups of 8 rows x 4 column phases unless groups of 32 rows alone fill the 16 warps
    if (r1 - r0 >= 512)
        mv_rowdots_rl<32, KIND, NV>(A, lda, r0, r1, ccap, xf, nv, red, out);
    else
        mv_rowdots_rl<8, KIND, NV>(A, lda, r0, r1, ccap, xf, nv, red, out);
}

// The products with the accumulator count fitted to nv (<= NVMAX): predicated-off FP64
// instructions would still take the FP64 pipe's issue slots.
template <int KIND, int NVMAX, class XF, class Out>
__device__ __forceinline__ void mv_rowdots(const double* __restrict__ A, int64_t lda, int64_t r0, int64_t r1,
                                           int64_t ccap, XF xf, int nv, double* red, Out out)
{
    if (r1 <= r0 || nv <= 0) return;
    if (nv <= NVMAX / 4)
        mv_rowdots_nv<KIND, NVMAX / 4>(A, lda, r0, r1, ccap, xf, nv, red, out);
    else if (nv <= NVMAX / 2)
        mv_rowdots_nv<KIND, NVMAX / 2>(A, lda, r0, r1, ccap, xf, nv, red, out);
    else
        mv_rowdots_nv<KIND, NVMAX>(A, lda, r0, r1, ccap, xf, nv, red, out);
}

template <int KIND, int NVMAX, class XF, class Out>
__device__ __forceinline__ void mv_coldots_fit(const double* __restrict__ A, int64_t lda, int64_t c0, int64_t c1,
                                               int64_t rlo, int64_t rhi, XF xf, int nv, double* red, Out out)
{
    if (nv <= NVMAX / 4)
        mv_coldots<KIND, NVMAX / 4>(A, lda, c0, c1, rlo, rhi, xf, nv, red, out);
    else if (nv <= NVMAX / 2)
        mv_coldots<KIND, NVMAX / 2>(A, lda, c0, c1, rlo, rhi, xf, nv, red, out);
    else
        mv_coldots<KIND, NVMAX>(A, lda, c0, c1, rlo, rhi, xf, nv, red, out);
}

// Sum over the team's ranks, in rank order, of the partial `idx` of each rank's block
// (ranks `stride` doubles apart); lane-strided, then a fixed xor tree.  Whole warp; every lane
// receives the result.
__device__ __forceinline__ double team_sum_at(const double* base, size_t stride, int G, size_t idx)
{
    const int lane = threadIdx.x & 31;
    double a = 0.0;
    for (int r = lane; r < G; r += 32) a += __ldcg(base + (size_t)r * stride + idx);
    return warp_sum(a);
}

// Teams at least this large sum the partials of S and of the Gram rows once per team (rank r
// a slice of the rows, then a team barrier) instead of on every CTA.
constexpr int kSliceBlock = 8;
// Fixed cost of a row of the T products (their lane-group reductions), in columns.
constexpr double kRowCost = 16.0;

// The team's sums of the partial rows [l0, l1) x nv (NB doubles per row, ranks `stride` apart,
// in rank order) written over rank 0's partials, rank `rank` summing its slice of the rows;
// returns after the team barrier that makes them visible (false: the barrier failed).
__device__ __forceinline__ bool reduce_rows(double* base, size_t stride, int G, int64_t l0, int64_t l1,
                                            int nv, int rank, Team& tm, int* err, uint32_t limit)
{
    const int64_t a = part_lo(l0, l1, rank, G), b = part_lo(l0, l1, rank + 1, G);
    for (int64_t q = threadIdx.x; q < (b - a) * nv; q += blockDim.x) {
        const int64_t l = a + q / nv;
        const int c = (int)(q % nv);
        const double v = sum_partials(base + l * kBlockMax + c, stride, G);
        base[l * kBlockMax + c] = v;
    }
    return team_sync(tm.bar, tm.target, G, err, limit);
}

// The block's staged vectors fit the shared-memory staging area.
__device__ __forceinline__ bool staging_fits(const Ws& w, int64_t mc, int nb)
{
    return (int64_t)2 * nb * mc <= w.xcap && (int64_t)nb * (mc + nb) <= w.xcap;
}

// Members per block the blocked path uses for a cluster of mc members on a team of G CTAs
// (1: the cluster takes the one-member path).
__device__ __forceinline__ int block_members(const Ws& w, int64_t mc, int G, int64_t n)
{
    if (w.block < 2 || mc < 3 || !w.vblk) return 1;
    // a CTA alone keeps the block's head rows in its own partial slot (16 n doubles), which
    // needs n >= 24; small problems stay with one member at a time
    if (G == 1 && n < 64) return 1;
    // up to 2 members per CTA (each CTA solves its members one after the other); the panel
    // buffer holds bb (n/G + 1) <= 2 n + 64 doubles
    // staged vectors in shared memory when they fit (nb doubles per row: 2 nb mc for the T
    // products, nb (mc + nb) for pass C), else read from the team's buffers in L2.  On a team a
    // CTA solves at most two members per sweep and holds its panel rows in shared memory; a CTA
    // alone solves them all and holds its panel in its q-vector buffer.
    const int nb = (G >= 2) ? min(w.block, 2 * G) : w.block;
    // the CTA-local solves use the staging area as their scratch
    if (w.xcap < SolveScratch<16>::size(1) || w.xcap < 6 * kStageRows) return 1;
    return nb;
}

// ---- one cluster by the blocked compact-WY path (Sec. 3.2; Alg. 4's sweeps per block) -----
__device__ __noinline__ bool bcwy_cluster(ChainCtx& cx, int32_t c, Team& tm, int nb)
{
    const Problem& p = cx.p;
    const Ws& w = cx.w;
    const int t = threadIdx.x, B = blockDim.x, wid = t >> 5, lane = t & 31, nW = B >> 5;
    const int G = tm.G, rank = tm.rank, leader = tm.leader;
    constexpr int NB = kBlockMax;
    const int64_t s0 = w.clstart[c];
    const int64_t mc = w.clsize[c];
    const JRef jr = jref(w, s0);
    const Seg& sg = *jr.g;
    const int64_t n = sg.n;
    double* Zc = p.Z + sg.z + jr.jl * sg.ldz;
    const int64_t ldz = sg.ldz;
    double* Tc = w.T + w.cltoff[c];
    const int64_t ldt = mc;
    double* Yc = w.Y + jr.off;
    const size_t ns = (size_t)p.n;
    const bool orth = (cx.mode == kModeOrth);
    const double onenrm = sg.onenrm, dtpcrt = sg.dtpcrt;
    const size_t pstride = 3 * (size_t)NB * ns;   // doubles of one CTA's partial block
    double* vb = w.vblk + (size_t)leader * NB * ns;  // member c's iterate at + c ns (all rows)
    double* qb = w.qblk + (size_t)leader * NB * ns;  // member c's q at + c ns (all rows)
    double* teamP = w.pblk + (size_t)leader * pstride;
    double* myP = teamP + (size_t)rank * pstride;
    double* pA = myP;                          // pass A partials [i NB + c]
    double* pG = myP + (size_t)NB * ns;        // Gram partials [i NB + c], rows k0.. hold Y_b^T Y_b
    double* pQ = myP + 2 * (size_t)NB * ns;    // panel and statistics partials (small)
    double* tb = w.tblk + (size_t)leader * pstride;
    double* sP = tb;                           // S' = T^T Y^T V  [i NB + c]
    double* tP = tb + (size_t)NB * ns;         // T_k (Y_k^T Y_b)  [i NB + c]
    double* xT = tb + 2 * (size_t)NB * ns;     // X_T, then T_k R1 before it  [i NB + c]
    // rows k0.. of Y_b [r NB + c]: in rank 1's slot of the team vectors, or, for a CTA alone,
    // after the panel and statistics partials of its own slot
    double* ybr = (G >= 2) ? tb + 3 * (size_t)NB * ns : pQ + 128;
    // this CTA's panel rows, column c at + c Rb: in shared memory on a team; a CTA alone holds
    // all rows k0.. of the panel in its q-vector buffer (free from the solves to pass C)
    double* W = (G >= 2) ? cx.vsm : qb;
    double* xs = cx.xs;                        // staged vectors, nbs doubles per row
    const int nbs = nb;
    // gst: the staged vectors are read from the team's buffers in L2 (they do not fit the
    // shared-memory staging area, which holds only small blocks); the team sums of S and the
    // Gram rows are then always formed by slices, so that they exist in global memory
    const bool gst = !staging_fits(w, mc, nb);
    const bool sliced = G >= kSliceBlock || gst;  // team sums of S and the Gram rows by slices
    double* red = cx.red;
    double* scal_t = w.partScal + (size_t)leader * kScalTeam;
    __shared__ double s_cv[NB], s_tv[NB], s_yh[NB], s_fac[NB], s_coef[NB];
    __shared__ double s_g22[NB * NB], s_t22[NB * NB], s_yb[NB * NB], s_stat[2 * NB];
    __shared__ int s_broke[NB], s_chk[NB];
    __shared__ int64_t s_rows[8];
    __shared__ double s_b[4];

    if (!TINV_IN(s0 >= 0 && mc >= 1 && s0 + mc <= w.nM && n <= p.n && rank < G && leader + G <= w.P &&
                     dbg_range((int64_t)jr.off, (int64_t)jr.off + mc * n, w.nF) &&
                     dbg_range(w.cltoff[c], w.cltoff[c] + mc * mc, w.nTT) &&
                     nb >= 2 && nb <= NB && (G == 1 || nb <= 2 * G) && (G >= 2 || (int64_t)NB * ns >= 384) &&
                     (p.zlen == 0 || dbg_range(sg.z + jr.jl * ldz, sg.z + (jr.jl + mc - 1) * ldz + n, p.zlen)),
                 cx.err))
        return false;

    const int64_t ra0 = part_lo(0, n, rank, G), ra1 = part_lo(0, n, rank + 1, G);
    int64_t kstart = 0;
    if (!orth) {
        // Alg. 4: Y_1 = [y_1], T_1 = [t_1] from the final head vector z
        const double* z = Zc;
        double ss = 0.0;
        for (int64_t r = ra0 + t; r < ra1; r += B) ss = fma(z[r], z[r], ss);
        ss = block_sum(ss, red);
        if (t == 0) scal_t[rank * kScalTeam + 6] = ss;
        if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
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
        if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
    }

    // blocks: stand-alone orthogonalization takes V's columns in order, nb at a time; inverse
    // iteration takes the members 1 + b + nblk c of block b
    const int64_t nblk = orth ? (mc + nb - 1) / nb : (mc - 1 + nb - 1) / nb;
    int64_t kpos = kstart;
    for (int64_t bi = 0; bi < nblk; ++bi) {
        const int64_t k0 = kpos;  // Y and T columns k0 .. k0 + bb - 1
        const int bb = (int)(orth ? min((int64_t)nb, mc - k0) : (mc - 1 - bi + nblk - 1) / nblk);
        kpos += bb;
        const int64_t kb = k0 + bb;
        const int64_t mem0 = orth ? k0 : 1 + bi;           // member of the block's column cc:
        const int64_t mstride = orth ? 1 : nblk;           //   mem0 + mstride cc
        if (t == 0) {
            s_rows[0] = part_lo(k0, n, rank, G);       // panel rows
            s_rows[1] = part_lo(k0, n, rank + 1, G);
            // rows of passes A and C: ranges of equal cost (a short row of the triangle costs
            // its length plus min(kb / 4, 128), the measured slowdown of short rows) when the largest
            // range (rank 0's) still lets pass A stage its V rows, equal rows otherwise
            const double c0 = fmin(0.25 * (double)kb, 128.0);
            const bool by_cost = (int64_t)bb * trap_row_lo(n, kb, 1, G, c0) <= 2 * n;
            s_rows[2] = trap_row_lo(n, kb, rank, G, by_cost ? c0 : -1.0);
            s_rows[3] = trap_row_lo(n, kb, rank + 1, G, by_cost ? c0 : -1.0);
            s_rows[4] = tri_col_lo(k0, rank, G);       // columns of T^T s
            s_rows[5] = tri_col_lo(k0, rank + 1, G);
            s_rows[6] = tri_row_lo_c(k0, rank, G, kRowCost);      // rows of the T products
            s_rows[7] = tri_row_lo_c(k0, rank + 1, G, kRowCost);
        }
        if (t < NB) s_chk[t] = 0;
        __syncthreads();
        const int64_t rb0 = s_rows[0], rb1 = s_rows[1], Rb = rb1 - rb0;
        const int64_t rc0 = s_rows[2], rc1 = s_rows[3];
        const int64_t c0 = s_rows[4], c1 = s_rows[5], i0 = s_rows[6], i1 = s_rows[7];
        if (!TINV_IN(dbg_range(rb0, rb1, n) && rb0 >= k0 && dbg_range(rc0, rc1, n) && dbg_range(c0, c1, k0) &&
                         dbg_range(i0, i1, k0) && (G == 1 || (int64_t)bb * Rb <= 2 * n + 64) && kb <= mc,
                     cx.err))
            return false;
        const int maxits = orth ? 1 : kMaxIts;
        int its = 0;
        while (its < maxits) {
            ++its;
            // ---- (S) the block's iterates: CTA-local solves, member cc on rank cc mod G ----
            XGlob vsrc{orth ? cx.V + k0 * cx.ldv : (its == 1 ? Zc + mem0 * ldz : vb),
                       orth ? cx.ldv : (its == 1 ? mstride * ldz : (int64_t)ns)};
            PROF_MARK(cx.prof, kPhEnd);
            if (!orth && its > 1) {
                for (int cc = rank; cc < bb; cc += G) {
                    const int64_t kk = mem0 + mstride * cc;
                    const Fac f = fac_at(w, jr.off + (size_t)kk * (size_t)n);
                    const bool may_end = s_chk[cc] >= kExtra || its == maxits;
                    uint32_t tgt = 0;
                    TeamRef tr{nullptr, &tgt, 1, 0, cx.err, nullptr, 0ull,
                               (unsigned long long*)&w.ctr[kCtrFallback],
                               may_end ? kSolveTol : kSolveTolLoose, 0u};
                    // all 16 warps of the CTA take chunks; the staging area is the scratch
                    if (!team_solve_nw<16>(n, f, qb + cc * ns, s_fac[cc], cx.vsm, vb + cc * ns, pG, 0, n,
                                           nullptr, nullptr, tr, xs))
                        return false;
                }
                PROF_MARK(cx.prof, kPhSolve);
                if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
                PROF_MARK(cx.prof, kPhLoad);
            }
            // ---- (A) partial S = Y_k^T V over this CTA's rows (V staged in shared memory when
            //      its rows fit the panel buffer) ----
            if (k0 > 0) {
                const int64_t Ra = rc1 - rc0;
                auto outA = [&](int64_t i, int cc, double v) { pA[i * NB + cc] = v; };
                if (G >= 2 && (int64_t)bb * Ra <= 2 * n) {
                    for (int64_t q = t; q < (int64_t)bb * Ra; q += B) {
                        const int cc = (int)(q / Ra);
                        W[q] = vsrc(rc0 + q % Ra, cc);
                    }
                    __syncthreads();
                    mv_coldots_fit<kLower, NB>(Yc, n, 0, k0, rc0, rc1, XCol{W, Ra, rc0}, bb, red, outA);
                } else {
                    mv_coldots_fit<kLower, NB>(Yc, n, 0, k0, rc0, rc1, vsrc, bb, red, outA);
                }
            }
            PROF_MARK(cx.prof, kPhA);
            if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhB1);
            // ---- (T1) S' = T_k^T S for the columns [c0, c1) of this CTA ----
            if (k0 > 0) {
                if (sliced) {  // S's rows summed once per team, rank r taking a slice of them
                    if (!reduce_rows(teamP, pstride, G, 0, k0, bb, rank, tm, cx.err, p.spin_limit))
                        return false;
                    if (!gst)
                        for (int64_t q = t; q < c1 * bb; q += B) {
                            const int64_t l = q / bb;
                            const int cc = (int)(q % bb);
                            xs[l * nbs + cc] = __ldcg(teamP + l * NB + cc);
                        }
                } else {
                    for (int64_t q = t; q < c1 * bb; q += B) {
                        const int64_t l = q / bb;
                        const int cc = (int)(q % bb);
                        xs[l * nbs + cc] = sum_partials(teamP + l * NB + cc, pstride, G);
                    }
                }
                __syncthreads();
                PROF_MARK(cx.prof, kPhT1a);
                auto outT1 = [&](int64_t i, int cc, double v) { sP[i * NB + cc] = v; };
                if (gst)
                    mv_coldots_fit<kUpper, NB>(Tc, ldt, c0, c1, 0, k0, XGRow{teamP, NB}, bb, red, outT1);
                else
                    mv_coldots_fit<kUpper, NB>(Tc, ldt, c0, c1, 0, k0, XRow{xs, nbs}, bb, red, outT1);
            }
            PROF_MARK(cx.prof, kPhT1);
            if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhB2);
            // ---- (B) panel rows of W = V - Y_k S' (this CTA's rows [rb0, rb1) of [k0, n)) ----
            if (k0 > 0 && !gst)
                for (int64_t q = t; q < k0 * bb; q += B) {
                    const int64_t l = q / bb;
                    const int cc = (int)(q % bb);
                    xs[l * nbs + cc] = __ldcg(&sP[l * NB + cc]);
                }
            for (int64_t q = t; q < (int64_t)bb * Rb; q += B) {
                const int cc = (int)(q / Rb);
                const int64_t r = rb0 + q % Rb;
                W[cc * Rb + (r - rb0)] = vsrc(r, cc);
            }
            __syncthreads();
            if (k0 > 0) {
                auto outB = [&](int64_t r, int cc, double v) { W[cc * Rb + (r - rb0)] -= v; };
                if (gst)
                    mv_rowdots<kAllCols, NB>(Yc, n, rb0, rb1, k0, XGRow{sP, NB}, bb, red, outB);
                else
                    mv_rowdots<kAllCols, NB>(Yc, n, rb0, rb1, k0, XRow{xs, nbs}, bb, red, outB);
            }
            PROF_MARK(cx.prof, kPhBb);
            // ---- (QR) Householder QR of the panel, one column (and team barrier) at a time ----
            for (int cc = 0; cc < bb; ++cc) {
                const int64_t col = k0 + cc;
                double* slot = pQ + (cc & 1) * 32;
                const int64_t lo = max(rb0, col);
                const double* wc = W + cc * Rb;
                // warp v: v = 0 the norm^2 of column cc, v > 0 its dot with column cc + v
                for (int v = wid; v < bb - cc; v += nW) {
                    const double* wv = W + (cc + v) * Rb;
                    double a = 0.0;
                    for (int64_t r = lo + lane; r < rb1; r += 32) a = fma(wc[r - rb0], wv[r - rb0], a);
                    a = warp_sum(a);
                    if (lane == 0) slot[v] = a;
                }
                // the head row's entries of columns cc.. (zero unless this CTA owns row col)
                if (t < bb - cc) slot[16 + t] = (col >= rb0 && col < rb1) ? W[(cc + t) * Rb + (col - rb0)] : 0.0;
                PROF_MARK(cx.prof, kPhB);
                if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
                PROF_MARK(cx.prof, kPhB3);
                // every CTA reduces the team's partials in rank order: identical decisions
                const size_t soff = 2 * (size_t)NB * ns + (cc & 1) * 32;
                for (int v = wid; v < 2 * (bb - cc); v += nW) {
                    const size_t idx = soff + (v < bb - cc ? v : 16 + (v - (bb - cc)));
                    const double s = team_sum_at(teamP, pstride, G, idx);
                    if (lane == 0) red[v] = s;
                }
                __syncthreads();
                if (wid == 0) {  // every lane forms the scalars (a warp costs what one lane does)
                    const double nrm = sqrt(red[0]);
                    const bool broke = !(nrm > 0.0) || !isfinite(nrm);
                    const double u1 = red[bb - cc];
                    const double cv = broke ? -1.0 : -sgn(u1) * nrm;
                    const double ue = broke ? 1.0 : u1;
                    const double tv = 1.0 / (cv * cv - ue * cv);
                    if (lane == 0) {
                        s_cv[cc] = cv;
                        s_tv[cc] = tv;
                        s_yh[cc] = ue - cv;
                        s_broke[cc] = broke ? 1 : 0;
                    }
                    // lane v: y^T w_{cc+v} = (w_cc - c e_col)^T w_{cc+v}, or 2 w_{cc+v}[col] after a
                    // breakdown
                    const int v = lane;
                    if (v >= 1 && v < bb - cc) {
                        const double hv = red[bb - cc + v];
                        s_coef[cc + v] = tv * (broke ? 2.0 * hv : red[v] - cv * hv);
                    }
                }
                __syncthreads();
                const bool broke = s_broke[cc] != 0;
                const double yh = s_yh[cc];
                // apply H_cc to the later columns of this CTA's rows, then make column cc the
                // reflector y (zero above row col) and store it as column col of Y
                for (int64_t q = t; q < Rb; q += B) {
                    const int64_t r = rb0 + q;
                    double yr = 0.0;
                    if (r >= col) yr = (r == col) ? yh : (broke ? 0.0 : W[cc * Rb + q]);
                    if (yr != 0.0)
                        for (int v = cc + 1; v < bb; ++v) W[v * Rb + q] = fma(-s_coef[v], yr, W[v * Rb + q]);
                    W[cc * Rb + q] = yr;
                    if (r >= col) Yc[r + col * n] = yr;
                }
                __syncthreads();
                PROF_MARK(cx.prof, kPhT2a);
            }
            // ---- (Gram) Y_k^T Y_b and Y_b^T Y_b over this CTA's panel rows; Y_b's rows k0.. ----
            if (k0 > 0)
                mv_coldots_fit<kLower, NB>(Yc, n, 0, k0, rb0, rb1, XCol{W, Rb, rb0}, bb, red,
                                       [&](int64_t i, int cc, double v) { pG[i * NB + cc] = v; });
            for (int v = wid; v < bb * bb; v += nW) {
                const int ca = v / bb, cb = v % bb;
                if (ca > cb) continue;  // upper triangle only
                double a = 0.0;
                for (int64_t q = lane; q < Rb; q += 32) a = fma(W[ca * Rb + q], W[cb * Rb + q], a);
                a = warp_sum(a);
                if (lane == 0) pG[(k0 + ca) * NB + cb] = a;
            }
            for (int64_t q = t; q < (int64_t)bb * bb; q += B) {
                const int64_t r = k0 + q / bb;
                const int cc = (int)(q % bb);
                if (r >= rb0 && r < rb1) ybr[(r - k0) * NB + cc] = W[cc * Rb + (r - rb0)];
            }
            PROF_MARK(cx.prof, kPhBc);
            if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhBa);
            // ---- (T2) T columns k0.. by Eq. cwy1 and X_T = T (rows col of Y) for pass C ----
            // Gram rows [0, k0 + bb): summed once per team by slices, or by every CTA
            double* gsum = teamP + NB * ns;  // rank 0's Gram partials, then the team's sums
            if (sliced && !reduce_rows(gsum, pstride, G, 0, k0 + bb, bb, rank, tm, cx.err, p.spin_limit))
                return false;
            auto gram = [&](int64_t l, int cc) {
                return sliced ? __ldcg(gsum + l * NB + cc) : sum_partials(gsum + l * NB + cc, pstride, G);
            };
            for (int v = t; v < bb * bb; v += B) {
                const int ca = v / bb, cb = v % bb;
                s_g22[ca * NB + cb] = (ca <= cb) ? gram(k0 + ca, cb) : 0.0;
                s_yb[ca * NB + cb] = __ldcg(&ybr[ca * NB + cb]);  // y_cb at row k0 + ca
            }
            // staged [G12 | R1] for the rows [i0, k0) of T_k, 2 nbs doubles per row (vector
            // v < bb: G12[l, v] = (Y_k^T Y_b)[l, v]; v = bb + c: R1[l, c] = Y[k0 + c, l], row
            // k0 + c of Y_k)
            if (!gst)
                for (int64_t q = t; q < (k0 - i0) * bb; q += B) {
                    const int64_t l = i0 + q / bb;
                    const int cc = (int)(q % bb);
                    xs[(l - i0) * 2 * nbs + cc] = gram(l, cc);
                    xs[(l - i0) * 2 * nbs + bb + cc] = __ldcg(&Yc[(k0 + cc) + l * n]);
                }
            __syncthreads();
            PROF_MARK(cx.prof, kPhT2b);
            // T_22 by the recurrence of Eq. cwy1 inside the block: T22[ca, cb] = -t_cb
            // sum_{ca <= l < cb} T22[ca, l] G22[l, cb] needs only row ca's earlier entries, so
            // lane ca of warp 0 takes row ca
            if (wid == 0 && lane < bb) {
                const int ca = lane;
                for (int cb = 0; cb < ca; ++cb) s_t22[ca * NB + cb] = 0.0;
                s_t22[ca * NB + ca] = s_tv[ca];
                for (int cb = ca + 1; cb < bb; ++cb) {
                    double a = 0.0;
                    for (int l = ca; l < cb; ++l) a = fma(s_t22[ca * NB + l], s_g22[l * NB + cb], a);
                    s_t22[ca * NB + cb] = -s_tv[cb] * a;
                }
            }
            // rows [i0, i1) of T_k times G12 (into tP) and times R1 (into xT)
            if (k0 > 0 && i1 > i0) {
                auto outP = [&](int64_t i, int v, double a) { tP[i * NB + v] = a; };
                auto outX = [&](int64_t i, int v, double a) { xT[i * NB + v] = a; };
                if (gst) {  // G12 from the team's sums, R1[l, c] = Y[k0 + c, l]
                    mv_rowdots<kUpperCol, NB>(Tc, ldt, i0, i1, k0, XGRow{gsum, NB}, bb, red, outP);
                    mv_rowdots<kUpperCol, NB>(Tc, ldt, i0, i1, k0, XGRow{Yc + k0, n}, bb, red, outX);
                } else {
                    const double* xg = xs - i0 * 2 * nbs;
                    mv_rowdots<kUpperCol, NB>(Tc, ldt, i0, i1, k0, XRow{xg, 2 * nbs}, bb, red, outP);
                    mv_rowdots<kUpperCol, NB>(Tc, ldt, i0, i1, k0, XRow{xg + bb, 2 * nbs}, bb, red, outX);
                }
            }
            __syncthreads();
            PROF_MARK(cx.prof, kPhT2c);
            // T_12 = -(T_k G12) T_22 (Eq. cwy1) for the rows [i0, i1), one entry per thread; the
            // rows are staged (xs is free again) for X_T[i, c] = (T_k R1)[i, c] +
            // sum_{c2 <= c} T[i, k0 + c2] y_c2[k0 + c]
            double* t12s = xs;
            for (int64_t q = t; q < (i1 - i0) * bb; q += B) {
                const int64_t i = i0 + q / bb;
                const int cc = (int)(q % bb);
                double a = 0.0;
                for (int l = 0; l <= cc; ++l) a = fma(__ldcg(&tP[i * NB + l]), s_t22[l * NB + cc], a);
                Tc[i + (k0 + cc) * ldt] = -a;
                if (!gst) t12s[(i - i0) * nbs + cc] = -a;
            }
            __syncthreads();
            for (int64_t q = t; q < (i1 - i0) * bb; q += B) {
                const int64_t i = i0 + q / bb;
                const int cc = (int)(q % bb);
                double a = __ldcg(&xT[i * NB + cc]);
                for (int c2 = 0; c2 <= cc; ++c2) {
                    const double t12 = gst ? __ldcg(&Tc[i + (k0 + c2) * ldt]) : t12s[(i - i0) * nbs + c2];
                    a = fma(t12, s_yb[cc * NB + c2], a);
                }
                xT[i * NB + cc] = a;
            }
            if (rank == 0 && t < bb * bb) {
                // the block's own rows: T_22 into T, X_T[k0 + ca, cb] = sum_{ca <= l <= cb} T_22[ca, l] y_l[k0 + cb]
                const int ca = t / bb, cb = t % bb;
                double a = 0.0;
                if (ca <= cb)
                    for (int l = ca; l <= cb; ++l) a = fma(s_t22[ca * NB + l], s_yb[cb * NB + l], a);
                xT[(k0 + ca) * NB + cb] = a;
                if (ca <= cb) Tc[(k0 + ca) + (k0 + cb) * ldt] = s_t22[ca * NB + cb];
            }
            PROF_MARK(cx.prof, kPhT2);
            if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhB4);
            // ---- (C) q_c = (Y T Y^T - I) e_{k0+c} = Y_{kb} X_T[:, c] - e_{k0+c}, rows [rc0, rc1) ----
            if (!gst)
                for (int64_t q = t; q < kb * bb; q += B) {
                    const int64_t l = q / bb;
                    const int cc = (int)(q % bb);
                    xs[l * nbs + cc] = __ldcg(&xT[l * NB + cc]);
                }
            __syncthreads();
            {
                auto outC = [&](int64_t r, int cc, double a) { qb[cc * ns + r] = (r == k0 + cc) ? a - 1.0 : a; };
                if (gst)
                    mv_rowdots<kLowerCol, NB>(Yc, n, rc0, rc1, kb, XGRow{xT, NB}, bb, red, outC);
                else
                    mv_rowdots<kLowerCol, NB>(Yc, n, rc0, rc1, kb, XRow{xs, nbs}, bb, red, outC);
            }
            // statistics of this CTA's rows: sum |q_c| (next scaling) and max |q_c| (the test)
            for (int cc = wid; cc < bb; cc += nW) {
                double as = 0.0;
                unsigned long long mb = 0;
                for (int64_t r = rc0 + lane; r < rc1; r += 32) {
                    const double x = qb[cc * ns + r];
                    as += fabs(x);
                    mb = max(mb, (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull);
                }
                as = warp_sum(as);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
                if (lane == 0) {
                    pQ[64 + cc] = as;
                    pQ[64 + NB + cc] = __longlong_as_double((long long)mb);
                }
            }
            PROF_MARK(cx.prof, kPhC);
            if (!team_sync(tm.bar, tm.target, G, cx.err, p.spin_limit)) return false;
            PROF_MARK(cx.prof, kPhB5);
            if (orth) {
                for (int cc = 0; cc < bb; ++cc)
                    for (int64_t r = ra0 + t; r < ra1; r += B) Zc[r + (k0 + cc) * ldz] = __ldcg(&qb[cc * ns + r]);
                break;
            }
            for (int v = wid; v < 2 * bb; v += nW) {
                const int cc = v % bb;
                const size_t idx = 2 * (size_t)NB * ns + 64 + (v < bb ? cc : NB + cc);
                double s;
                if (v < bb) {
                    s = team_sum_at(teamP, pstride, G, idx);
                } else {
                    unsigned long long mb = 0;
                    for (int r = lane; r < G; r += 32)
                        mb = max(mb, (unsigned long long)__double_as_longlong(__ldcg(teamP + (size_t)r * pstride + idx)));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
                    s = __longlong_as_double((long long)mb);
                }
                if (lane == 0) s_stat[v < bb ? cc : NB + cc] = s;
            }
            __syncthreads();
            // convergence test on x_c = -c_c q_c (||x||_inf = |c_c| max|q_c|), per member
            if (wid == 0) {  // lane cc tests member cc
                const int cc = lane;
                bool done = true;
                if (cc < bb) {
                    if (!s_broke[cc] && fabs(s_cv[cc]) * s_stat[NB + cc] >= dtpcrt) ++s_chk[cc];
                    done = s_chk[cc] >= kExtra + 1;
                    const int64_t j = s0 + mem0 + mstride * cc;
                    s_fac[cc] = -sgn(s_cv[cc]) * (((double)n * onenrm) * fmax(kEps, w.u0n[j])) / s_stat[cc];
                }
                const bool all = __all_sync(0xffffffffu, done);
                if (lane == 0) s_b[3] = all ? 1.0 : 0.0;
            }
            __syncthreads();
            if (s_b[3] != 0.0 || its == maxits) {
                // Alg. 4's normalization and sign are applied by k_finalize
                for (int cc = 0; cc < bb; ++cc)
                    for (int64_t r = ra0 + t; r < ra1; r += B)
                        Zc[r + (mem0 + mstride * cc) * ldz] = __ldcg(&qb[cc * ns + r]);
                if (rank == 0 && t < bb) {
                    const int64_t j = s0 + mem0 + mstride * t;
                    const bool conv = s_chk[t] >= kExtra + 1;
                    if (p.iters) p.iters[j] = conv ? its : -its;
                    if (!conv) count_nonconverged(w, j);
                }
                break;
            }
        }
        // Y's block columns and T are complete (last barrier); Z rows are written per CTA
        __syncthreads();
    }
    return true;
}
