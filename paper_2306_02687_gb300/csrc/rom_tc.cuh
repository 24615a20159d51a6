// rom_tc.cuh -- mixed-precision evaluation kernel whose reduced-tangent
// contraction (step a5, Eqs. ROMstiffness and Biot_Tangent of Sec. 3.2) runs
// on the tcgen05 tensor cores.
//
// The augmented system of one macro point alpha,
//     M_alpha = sum_i Bext_i^T Y_i,  Y_i = w_i A_i Bext_i,  Bext_i = [B_i | I],
// is computed for all points of a CTA at once as one matrix product whose
// shared operand is the gradient table:
//     D[(alpha, j), c] = sum_k Y[k, (alpha, j)] Bext[k, c],   k = (i, component)
// A operand: the Y rows of the CTA's points stacked along M (16 or 32 rows
//            per point, one 128-row MMA tile per warp), built in shared
//            memory per k-step of 8.
// Work split: each warp owns one tile (PPT points) for the whole ECM loop:
// it evaluates the law for its points, builds its A rows, issues and commits
// its own MMAs and accumulates its points' residual, so a k-step needs only
// warp-level synchronization; the only CTA barrier per chunk of ECM points
// comes with the fold of the TMEM accumulators, where a warp reads one lane
// quarter of every tile.
// B operand: Bext, pre-split on the host into TF32 leading and trailing parts
//            and pre-arranged in the MMA's core-matrix layout, so that a chunk
//            of ECM points is one contiguous bulk (TMA) copy.
// Precision: three TF32 products per k-step (Yhi Bhi + Yhi Blo + Ylo Bhi)
// give float32-level products; the tensor core's float32 accumulation (which
// does not round to nearest) runs over one chunk of CI ECM points only, and
// the chunk sums are added into a running sum (also in TMEM) with Kahan
// compensation, like the compensated chunk sums of the SIMT kernel.
// Steps a1-a4 are the mixed form of the SIMT kernel (double-float
// kinematics, law, residual and homogenized stress; float32 tangent).  The
// kernel ends with a per-point workspace record (the augmented system, the
// right-hand side, the micro state, the polar factors); condense_kernel
// then performs steps a6 and a7 with one thread per point.
#pragma once

#include "rom_condense.cuh"
#include "rom_core.cuh"
#include "tc.cuh"

namespace rverom {

constexpr int ST_TIMEOUT = 5;  // an internal wait of the kernel ran out (outputs invalid)

__host__ __device__ constexpr size_t tc_al(size_t x) { return (x + 127) / 128 * 128; }

template <int D, int NA, int NP, int CI>
struct TcPlan {
    static constexpr int G = D * D;
    static constexpr int NS = Dims<D>::NS;
    static constexpr int NQ = NA - G;
    static constexpr int QP = NQ | 1;
    static constexpr int BP = NQ | 1;
    static constexpr int NAR = NA <= 16 ? 16 : 32;  // A-operand rows per point
    static constexpr int PPT = 128 / NAR;           // points per 128-row tile
    static constexpr int NN = (NA + 15) / 16 * 16;  // MMA N (columns of Bext)
    static constexpr int NT = 256;
    static constexpr int NW = NT / 32;              // warps = tiles
    static constexpr int EPS = 8 / G;               // ECM points per k-step of 8
    static constexpr int KSC = CI / EPS;            // k-steps per chunk
    static constexpr int RPW = (PPT * NQ + 31) / 32;  // residual outputs per lane
    static constexpr int TCOLS = 2 * NW * NN;       // accumulator + running sum
    static constexpr int TALLOC = TCOLS <= 32 ? 32 : TCOLS <= 64 ? 64 : TCOLS <= 128 ? 128 : TCOLS <= 256 ? 256 : 512;
    static_assert(D == 2, "planar RVEs (two ECM points per k-step)");
    static_assert(NA <= 32, "register-resident condensation");
    static_assert(NP == NW * PPT, "one tile per warp");
    static_assert(CI * PPT == 32, "one law evaluation per lane and chunk");
    static_assert(CI % EPS == 0, "a chunk holds whole k-steps");
    static_assert(TCOLS <= 512, "TMEM holds 512 columns");
    // byte offsets
    static constexpr size_t YWARP = 4 * 4096;  // per warp: [2 buffers][hi|lo][2 kg][16 rg][8][4] floats
    static constexpr size_t o_Y = 0;
    static constexpr size_t BXPART = (size_t)NN * 32;  // [NN/8][2 kg][8][4] floats
    static constexpr size_t BXBUF = (size_t)KSC * 2 * BXPART;
    static constexpr size_t o_BX = tc_al(o_Y + NW * YWARP);
    static constexpr size_t NBST = (size_t)CI * G * BP;  // (hi, lo) pairs per staging buffer
    static constexpr size_t o_B = tc_al(o_BX + 2 * BXBUF);
    static constexpr size_t o_w = tc_al(o_B + 2 * 2 * NBST * 4);
    static constexpr size_t o_ph = tc_al(o_w + 2 * 2 * CI * 4);
    static constexpr size_t o_W = tc_al(o_ph + 2 * CI * 4);            // [warp][il][p][G*G]
    static constexpr size_t o_WP = tc_al(o_W + (size_t)NP * CI * G * G * 4);  // (hi, lo): [warp][il][c][p]
    static constexpr size_t o_q = tc_al(o_WP + 2 * (size_t)NP * CI * G * 4);
    static constexpr size_t o_q64 = tc_al(o_q + 2 * (size_t)NP * QP * 4);
    static constexpr size_t o_U = tc_al(o_q64 + (size_t)NP * QP * 8);
    static constexpr size_t o_R = tc_al(o_U + (size_t)NP * G * 8);
    static constexpr size_t o_dU = tc_al(o_R + (size_t)NP * G * 8);
    static constexpr size_t o_Udf = tc_al(o_dU + (size_t)NP * NS * 8);
    static constexpr size_t o_flag = tc_al(o_Udf + 2 * (size_t)NP * G * 4);
    static constexpr size_t o_pidx = o_flag + NP * 4;
    // mbarriers: [0,1] table copies, [2 + 2 w + b] MMA commits of warp w per
    // A buffer, [2 + 2 NW + w] MMAs of a whole chunk of warp w; then TMEM
    // slot, error flag
    static constexpr size_t o_bar = tc_al(o_pidx + NP * 4);
    // mbarriers: bx[2], commit[NW][2], chunk[NW], drain
    static constexpr size_t o_slot = o_bar + (3 + 3 * NW) * 8;
    static constexpr size_t bytes = tc_al(o_slot + 8);
    static_assert(bytes <= 227 * 1024, "shared memory");
};

// Bext image for the B operand: per k-step of 8 (k = i * G + c), the TF32
// leading part then the trailing part, each [nn/8][2][8][4] floats (built by
// the host when the ROM is loaded).
template <int D, int NA, int NP, int CI>
__global__ void __launch_bounds__(256, 1) eval_tc_kernel(EvalArgs a) {
    using PL = TcPlan<D, NA, NP, CI>;
    constexpr int G = PL::G, NS = PL::NS, NQ = PL::NQ, QP = PL::QP, BP = PL::BP;
    constexpr int NAR = PL::NAR, PPT = PL::PPT, NN = PL::NN, NW = PL::NW;
    constexpr int EPS = PL::EPS, KSC = PL::KSC, NT = PL::NT, RPW = PL::RPW;
    constexpr int NBST = (int)PL::NBST;
    using CR = CondRec<D, NA>;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_BX = reinterpret_cast<float *>(smem + PL::o_BX);
    float2 *s_Bst = reinterpret_cast<float2 *>(smem + PL::o_B);  // (hi, lo) of the B table: [buf][il * G + c][BP]
    float *s_wst = reinterpret_cast<float *>(smem + PL::o_w);
    int *s_ph = reinterpret_cast<int *>(smem + PL::o_ph);
    float2 *s_q2 = reinterpret_cast<float2 *>(smem + PL::o_q);  // (hi, lo) of q: [p][QP]
    double *s_qd = reinterpret_cast<double *>(smem + PL::o_q64);
    double *s_U = reinterpret_cast<double *>(smem + PL::o_U);
    double *s_R = reinterpret_cast<double *>(smem + PL::o_R);
    double *s_dU = reinterpret_cast<double *>(smem + PL::o_dU);
    float *s_Uh = reinterpret_cast<float *>(smem + PL::o_Udf), *s_Ul = s_Uh + NP * G;
    int *s_flag = reinterpret_cast<int *>(smem + PL::o_flag);
    int *s_pidx = reinterpret_cast<int *>(smem + PL::o_pidx);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + PL::o_bar);
    uint32_t *s_slot = reinterpret_cast<uint32_t *>(smem + PL::o_slot);
    volatile int *s_err = reinterpret_cast<volatile int *>(smem + PL::o_slot + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.t.n, m = a.t.m;
    const int na = n + G;
    const int64_t count = a.count ? (int64_t)(*a.count) : a.n_points;
    const int64_t off = (a.perm && a.offset) ? (int64_t)(*a.offset) : 0;
    const int32_t *perm = a.perm ? a.perm + off : nullptr;
    float *ws = a.cond + off * CR::W;  // records of this type's points, by list position
    // this CTA's share of the list: a contiguous range (shares differ by at
    // most one point), taken in tiles of NP points with a partial last tile
    // whose missing points cost (almost) nothing
    const int64_t r_begin = count * blockIdx.x / gridDim.x, r_end = count * (blockIdx.x + 1) / gridDim.x;
    const int nch = (m + CI - 1) / CI;
    // this warp's tile: points p0 .. p0 + PPT - 1 of the CTA, its A rows, its
    // TMEM accumulator columns, its MMA commit barriers
    const int p0 = warp * PPT;
    float *yw = reinterpret_cast<float *>(smem + PL::o_Y + warp * PL::YWARP);
    float *Ww = reinterpret_cast<float *>(smem + PL::o_W) + warp * CI * PPT * G * G;
    float2 *WP2 = reinterpret_cast<float2 *>(smem + PL::o_WP) + warp * CI * G * PPT;  // (hi, lo) of w_i P_i
    uint64_t *mbar = s_bar + 2 + 2 * warp;

    const df dmu0 = df_from(a.t.mu[0]), dmu1 = df_from(a.t.mu[1]);
    const df dlam0 = df_from(a.t.kappa[0] - (2.0 / 3.0) * a.t.mu[0]);
    const df dlam1 = df_from(a.t.kappa[1] - (2.0 / 3.0) * a.t.mu[1]);
    const float kmu0 = (float)a.t.mu[0], kmu1 = (float)a.t.mu[1];
    const float klam0 = (float)(a.t.kappa[0] - (2.0 / 3.0) * a.t.mu[0]);
    const float klam1 = (float)(a.t.kappa[1] - (2.0 / 3.0) * a.t.mu[1]);

    if (warp == 0) {
        tc::tmem_alloc(s_slot, PL::TALLOC);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2 + 3 * NW; ++b) tc::mbar_init(&s_bar[b], 1);
        tc::mbar_init(&s_bar[2 + 3 * NW], NW);  // drain
        tc::mbar_init_fence();
        *s_err = 0;
    }
    // staging buffers: zero once (entries past m keep finite values); the
    // A-operand buffers too (a warp without points in a tile leaves them as
    // they are, and its MMAs read them)
    for (int x = tid; x < 2 * NBST; x += NT) s_Bst[x] = make_float2(0.0f, 0.0f);
    for (int x = tid; x < (int)(NW * PL::YWARP / 4); x += NT) reinterpret_cast<float *>(smem + PL::o_Y)[x] = 0.0f;
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *s_slot;
    const uint32_t idesc = tc::idesc_tf32(128, NN);
    // bounded wait (tc::WAIT_LIMIT_NS); after the first timeout no wait
    // blocks any more, no MMA or bulk copy is issued, and the tile's points
    // are marked ST_TIMEOUT
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*s_err == 0 && !tc::mbar_wait(bar, parity)) *s_err = 1;
    };
    uint32_t gstep = 0, gchunk = 0;  // k-steps and chunks issued by this CTA so far

    auto stage_cp = [&](int buf, int i0s) {
        float *b2 = reinterpret_cast<float *>(s_Bst + buf * NBST);
        float *wh = s_wst + buf * 2 * CI, *wl = wh + CI;
        const int cnt = min(CI, m - i0s) * G * n;
        for (int x = tid; x < cnt; x += NT) {
            const int r = x / n, j = x - r * n;  // r = il * G + c
            const int64_t gi = (int64_t)i0s * G * n + x;
            cp_async4(b2 + 2 * (r * BP + j), a.t.Bh + gi);
            cp_async4(b2 + 2 * (r * BP + j) + 1, a.t.Bl + gi);
        }
        if (tid < min(CI, m - i0s)) {
            cp_async4(wh + tid, a.t.wh + i0s + tid);
            cp_async4(wl + tid, a.t.wl + i0s + tid);
            cp_async4(s_ph + buf * CI + tid, a.t.phase + i0s + tid);
        }
        cp_async_commit();
    };
    // bulk copy of the B-operand image of chunk ch (CTA-wide chunk index g)
    // into buffer g & 1, by one thread; nothing is issued once a wait of the
    // CTA has timed out
    int64_t bx_last0 = -1, bx_last1 = -1;  // last chunk index copied into each buffer (thread 0)
    auto stage_bulk = [&](uint32_t g, int ch) {
        if (*s_err != 0) return;
        const int buf = g & 1;
        if (buf) bx_last1 = g; else bx_last0 = g;
        tc::mbar_arrive_expect_tx(&s_bar[buf], (uint32_t)PL::BXBUF);
        tc::bulk_g2s(s_BX + buf * (PL::BXBUF / 4), a.t.Bimg + (size_t)ch * (PL::BXBUF / 4), (uint32_t)PL::BXBUF,
                     &s_bar[buf]);
    };

    for (int64_t t0 = r_begin; t0 < r_end; t0 += NP) {
        const int nlive = (int)min((int64_t)NP, r_end - t0);  // points of this tile
        const bool wlive = p0 < nlive;                         // this warp's tile holds points
        // ---- a1: polar split, micro update ---------------------------------
        if (tid < NP) {
            const int p = tid;
            const int64_t li = t0 + p;
            int gp = -1;
            if (p < nlive) gp = perm ? perm[li] : (int)li;
            s_pidx[p] = gp;
            int flag = -1;
            double F[G], R[G], U[G];
            if (gp >= 0) {
                flag = ST_OK;
                bool fin = true;
#pragma unroll
                for (int c = 0; c < G; ++c) {
                    F[c] = a.Fbar[(int64_t)gp * G + c];
                    fin = fin && isfinite(F[c]);
                }
                if (!fin) flag = ST_NONFINITE;
                else if (!(det<D>(F) > 0.0) || !polar<D>(F, R, U)) flag = ST_DETF;
            }
            if (flag != ST_OK) {
#pragma unroll
                for (int c = 0; c < G; ++c) {
                    R[c] = (c % (D + 1) == 0) ? 1.0 : 0.0;
                    U[c] = R[c];
                }
            }
#pragma unroll
            for (int c = 0; c < G; ++c) {
                s_U[p * G + c] = U[c];
                s_R[p * G + c] = R[c];
                const df u = df_from(U[c]);
                s_Uh[p * G + c] = u.hi;
                s_Ul[p * G + c] = u.lo;
            }
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                int i, j;
                voigt_pair(D, v, i, j);
                s_dU[p * NS + v] = (flag == ST_OK) ? U[i * D + j] - a.Uprev[(int64_t)gp * NS + v] : 0.0;
            }
            s_flag[p] = flag;
        }
        __syncthreads();
        for (int x = tid; x < NP * NQ; x += NT) {
            const int p = x / NQ, j = x % NQ;
            const int gp = s_pidx[p];
            double qv = 0.0;
            if (j < n && gp >= 0 && s_flag[p] == ST_OK) {
                const int64_t base = (int64_t)gp * a.nmax + j;
                qv = a.q[base] - a.s[base];
#pragma unroll
                for (int v = 0; v < NS; ++v) qv -= a.S[base * NS + v] * s_dU[p * NS + v];
            }
            s_qd[p * QP + j] = qv;
            const df v = df_from(qv);
            s_q2[p * QP + j] = make_float2(v.hi, v.lo);
        }
        dacc rdacc[2 * RPW];
#pragma unroll
        for (int u = 0; u < 2 * RPW; ++u) rdacc[u] = dacc{0.0f, 0.0f};
        df pudf{0.0f, 0.0f};
        // first chunk's tables
        stage_cp(gchunk & 1, 0);
        if (tid == 0) stage_bulk(gchunk, 0);
        cp_async_wait<0>();
        __syncthreads();

        // ---- ECM loop: a2-a5 ----------------------------------------------
        int folds = 0;
        for (int ch = 0; ch < nch; ++ch, ++gchunk) {
            const int buf = gchunk & 1;
            const int i0 = ch * CI;
            // prefetch the next chunk: its staging buffer and table image were
            // last read in chunk ch-1, which every warp finished (the MMAs too)
            // before the barrier that closed it
            if (ch + 1 < nch) {
                stage_cp(buf ^ 1, i0 + CI);
                if (tid == 0) stage_bulk(gchunk + 1, ch + 1);
            }
            const float2 *B2 = s_Bst + buf * NBST;
            const float *wh = s_wst + buf * 2 * CI, *wl = wh + CI;

            // pointwise (this warp's points, one ECM point per lane):
            // F_i, law, w P_i (double-float), W_i = w_i A_i (float32)
            {
                const int pl = lane % PPT, il = lane / PPT;
                const int p = p0 + pl;
                bool live = (s_flag[p] == ST_OK) && (i0 + il < m);
                const int ph = s_ph[buf * CI + il];
                float fi[G];
                float lnJk = 0.0f;
                if (live) {
                    df F[G], P[G];
                    const float2 *b2 = B2 + il * G * BP;
                    const float2 *q2 = s_q2 + p * QP;
                    dacc sacc[G];
#pragma unroll
                    for (int c = 0; c < G; ++c) sacc[c] = dacc{s_Uh[p * G + c], s_Ul[p * G + c]};
#pragma unroll 4
                    for (int j = 0; j < n; ++j) {
                        const float2 qj = q2[j];
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            const float2 bj = b2[c * BP + j];
                            dacc_fma(sacc[c], bj.x, bj.y, qj.x, qj.y);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < G; ++c) F[c] = dacc_get(sacc[c]);
                    if (!nh_stress_df<D>(F, ph ? dmu1 : dmu0, ph ? dlam1 : dlam0, P, fi, lnJk)) {
                        atomicCAS(&s_flag[p], ST_OK, ST_DETF);
                        live = false;
                    } else {
                        const df w2{wh[il], wl[il]};
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            const df wp = df_mul(w2, P[c]);
                            WP2[(il * G + c) * PPT + pl] = make_float2(wp.hi, wp.lo);
                        }
                    }
                }
                float4 *Wt = reinterpret_cast<float4 *>(Ww + (il * PPT + pl) * G * G);
                if (live) {
                    const float muk = ph ? kmu1 : kmu0, lam = ph ? klam1 : klam0;
                    const float c3 = muk - lam * lnJk;
                    const float wk = wh[il];
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        float Ar[G];
                        nh_tangent_row<D, float>(fi, lam, c3, muk, c, Ar);
                        Wt[c] = make_float4(wk * Ar[0], wk * Ar[1], wk * Ar[2], wk * Ar[3]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        WP2[(il * G + c) * PPT + pl] = make_float2(0.0f, 0.0f);
                        Wt[c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
                }
            }
            __syncwarp();

            // a5: per k-step, this warp builds its tile's A rows and issues
            // its three MMAs (D_tile += Yhi Bhi + Yhi Blo + Ylo Bhi)
            const int j = lane % NAR;  // row within the point (the same for all of this lane's rows)
            for (int ks = 0; ks < KSC; ++ks) {
                const uint32_t s = gstep + ks;
                const int yb = s & 1;
                if (s >= 2) wait(&mbar[yb], ((s - 2) >> 1) & 1);
                float *Yh = yw + yb * 2048, *Yl = Yh + 1024;
#pragma unroll
                for (int e = 0; e < EPS; ++e) {
                    if (!wlive) break;
                    const int il = ks * EPS + e;
                    float bx[G];
#pragma unroll
                    for (int d = 0; d < G; ++d) bx[d] = (j < n) ? B2[(il * G + d) * BP + j].x : ((j - n == d) ? 1.0f : 0.0f);
                    const bool jin = j < na;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int rl = k * 32 + lane;  // row within the tile
                        const int pl = rl / NAR;
                        const float4 *Wt = reinterpret_cast<const float4 *>(Ww + (il * PPT + pl) * G * G);
                        float y[G];
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            const float4 wv = Wt[c];
                            float v = wv.x * bx[0];
                            v = __fmaf_rn(wv.y, bx[1], v);
                            v = __fmaf_rn(wv.z, bx[2], v);
                            v = __fmaf_rn(wv.w, bx[3], v);
                            y[c] = jin ? v : 0.0f;
                        }
                        float hi[G], lo[G];
#pragma unroll
                        for (int c = 0; c < G; ++c) tc::split_tf32(y[c], hi[c], lo[c]);
                        const int off = e * 512 + rl * 4;
                        *reinterpret_cast<float4 *>(Yh + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                        *reinterpret_cast<float4 *>(Yl + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                    }
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0 && ks == 0) wait(&s_bar[buf], (gchunk >> 1) & 1);
                if (lane == 0 && *s_err == 0) {
                    tc::fence_after_sync();
                    const uint32_t ba = tc::smem_u32(s_BX + buf * (PL::BXBUF / 4) + ks * 2 * (PL::BXPART / 4));
                    const uint64_t bdh = tc::smem_desc(ba, 128, 256);
                    const uint64_t bdl = tc::smem_desc(ba + (uint32_t)PL::BXPART, 128, 256);
                    const uint64_t adh = tc::smem_desc(tc::smem_u32(Yh), 2048, 128);
                    const uint64_t adl = tc::smem_desc(tc::smem_u32(Yl), 2048, 128);
                    const uint32_t dt = tbase + warp * NN;
                    // a chunk's first MMA starts the accumulator fresh in the first
                    // two chunks; later it adds onto the fold's compensation term
                    tc::mma_tf32(dt, adh, bdh, idesc, (ks > 0 || ch >= 2) ? 1u : 0u);
                    tc::mma_tf32(dt, adh, bdl, idesc, 1u);
                    tc::mma_tf32(dt, adl, bdh, idesc, 1u);
                    tc::mma_commit(&mbar[yb]);
                    if (ks == KSC - 1) tc::mma_commit(&s_bar[2 + 2 * NW + warp]);  // the whole chunk
                }
                __syncwarp();
            }
            gstep += KSC;

            // a4: float64-accurate reduced residual and homogenized stress of
            // this warp's points
            // all of this lane's rows at once (2 RPW independent chains); a row
            // past the warp's points reads row 0 and is never stored, and rows
            // j >= n are stored as zero
            if (wlive) {
                int bo[RPW], wo[RPW];
#pragma unroll
                for (int u = 0; u < RPW; ++u) {
                    const int o = lane + 32 * u;
                    const bool in = o < PPT * NQ;
                    wo[u] = in ? o / NQ : 0;
                    bo[u] = in ? o % NQ : 0;
                }
#pragma unroll
                for (int il = 0; il < CI; il += 2)
#pragma unroll
                    for (int c = 0; c < G; ++c)
#pragma unroll
                        for (int u = 0; u < RPW; ++u) {
                            const int b0 = (il * G + c) * BP + bo[u], w0 = (il * G + c) * PPT + wo[u];
                            const int b1 = b0 + G * BP, w1 = w0 + G * PPT;
                            const float2 x0 = B2[b0], y0 = WP2[w0], x1 = B2[b1], y1 = WP2[w1];
                            dacc_fma(rdacc[2 * u], x0.x, x0.y, y0.x, y0.y);
                            dacc_fma(rdacc[2 * u + 1], x1.x, x1.y, y1.x, y1.y);
                        }
            }
            if (lane < PPT * G) {
                const int pl = lane / G, c = lane % G;
                for (int il = 0; il < CI; ++il) {
                    const float2 v = WP2[(il * G + c) * PPT + pl];
                    pudf = df_add(pudf, df{v.x, v.y});
                }
            }

            // fold the chunk accumulators into the running sums (TMEM), Kahan-
            // compensated: the compensation term is stored (negated) into the
            // accumulator, onto which the next chunk's MMAs add, so the next
            // fold adds (chunk sum - compensation).  The last fold writes the
            // augmented system of every point to the workspace.  A warp reads
            // its lane quarter of every other tile, so it waits for the chunk
            // barrier of every warp: one phase per chunk, so the phase waited
            // for is always the barrier's current one or the one before it (a
            // parity wait is defined only for those two; the per-buffer
            // barriers advance twice per chunk and would not do).
            const bool last = (ch == nch - 1);
            {
                for (int w2 = 0; w2 < NW; ++w2)
                    wait(&s_bar[2 + 2 * NW + w2], gchunk & 1);
                __syncwarp();  // the TMEM loads below are warp-collective
                tc::fence_after_sync();
                const int qd = warp & 3;
                const uint32_t lanes = (uint32_t)(qd * 32) << 16;
                for (int t = warp >> 2; t < NW; t += 2) {
                    if (t * PPT >= nlive) break;  // tiles without points (their rows are never read)
                    const int row = t * 128 + qd * 32 + lane;
                    const int p = row / NAR, jr = row % NAR;
#pragma unroll
                    for (int cb = 0; cb < NN / 32; ++cb) {
                        float va[32], vs[32];
                        tc::tmem_ld32(tbase + lanes + t * NN + cb * 32, va);
                        if (folds > 0) tc::tmem_ld32(tbase + lanes + NW * NN + t * NN + cb * 32, vs);
                        tc::tmem_wait_ld();
                        if (folds > 0) {
#pragma unroll
                            for (int c = 0; c < 32; ++c) {
                                const float tt = __fadd_rn(vs[c], va[c]);
                                vs[c] = __fsub_rn(va[c], __fsub_rn(tt, vs[c]));  // -(compensation)
                                va[c] = tt;
                            }
                            if (!last) tc::tmem_st32(tbase + lanes + t * NN + cb * 32, vs);
                        }
                        if (!last) {
                            tc::tmem_st32(tbase + lanes + NW * NN + t * NN + cb * 32, va);
                        } else if (jr < NA && p < nlive) {
                            // lane jr holds column jr of M: entries (col, jr), col >= jr
                            float *rm = ws + (t0 + p) * CR::W + CR::o_M;
#pragma unroll
                            for (int c = 0; c < 32; ++c) {
                                const int col = cb * 32 + c;
                                if (col < NA && col >= jr) rm[tri(col, jr)] = va[c];
                            }
                        }
                    }
                    if (NN % 32) {
                        constexpr int cb = NN / 32;
                        float va[16], vs[16];
                        tc::tmem_ld16(tbase + lanes + t * NN + cb * 32, va);
                        if (folds > 0) tc::tmem_ld16(tbase + lanes + NW * NN + t * NN + cb * 32, vs);
                        tc::tmem_wait_ld();
                        if (folds > 0) {
#pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const float tt = __fadd_rn(vs[c], va[c]);
                                vs[c] = __fsub_rn(va[c], __fsub_rn(tt, vs[c]));
                                va[c] = tt;
                            }
                            if (!last) tc::tmem_st16(tbase + lanes + t * NN + cb * 32, vs);
                        }
                        if (!last) {
                            tc::tmem_st16(tbase + lanes + NW * NN + t * NN + cb * 32, va);
                        } else if (jr < NA && p < nlive) {
                            float *rm = ws + (t0 + p) * CR::W + CR::o_M;
#pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const int col = cb * 32 + c;
                                if (col < NA && col >= jr) rm[tri(col, jr)] = va[c];
                            }
                        }
                    }
                }
                if (!last) tc::tmem_wait_st();
                ++folds;
            }
            tc::fence_before_sync();
            if (ch + 1 < nch) cp_async_wait<0>();
            __syncthreads();
            tc::fence_after_sync();
        }

        // ---- workspace records of this warp's points (steps a6, a7 follow in
        // condense_kernel): residual and V0 Pbar_U (double-float), q, R, U, status
        const int err = *s_err;
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
            const int o = lane + 32 * u;
            if (o < PPT * NQ) {
                const int pl = o / NQ, jj = o % NQ;
                const int64_t li = t0 + p0 + pl;
                if (p0 + pl < nlive) {
                    const df v = jj < n ? df_add(dacc_get(rdacc[2 * u]), dacc_get(rdacc[2 * u + 1])) : df{0.0f, 0.0f};
                    float *rec = ws + li * CR::W;
                    rec[CR::o_rh + jj] = v.hi;
                    rec[CR::o_rl + jj] = v.lo;
                    reinterpret_cast<double *>(rec + CR::o_q)[jj] = s_qd[(p0 + pl) * QP + jj];
                }
            }
        }
        if (lane < PPT * G) {
            const int pl = lane / G, c = lane % G;
            const int64_t li = t0 + p0 + pl;
            if (p0 + pl < nlive) {
                float *rec = ws + li * CR::W;
                rec[CR::o_ph + c] = pudf.hi;
                rec[CR::o_pl + c] = pudf.lo;
                reinterpret_cast<double *>(rec + CR::o_R)[c] = s_R[(p0 + pl) * G + c];
                reinterpret_cast<double *>(rec + CR::o_U)[c] = s_U[(p0 + pl) * G + c];
                if (c == 0) *reinterpret_cast<int *>(rec + CR::o_flag) = err ? ST_TIMEOUT : s_flag[p0 + pl];
            }
        }
        __syncthreads();
    }
    // drain before TMEM is freed: every MMA this warp issued has completed
    // (immediate unless a timeout skipped the fold waits), and the last bulk
    // copy into each buffer has landed
    if (lane == 0) {
        tc::mma_commit(&s_bar[2 + 3 * NW]);
        tc::mbar_wait(&s_bar[2 + 3 * NW], 0);
    }
    if (tid == 0) {
        if (bx_last0 >= 0) tc::mbar_wait(&s_bar[0], (uint32_t)(bx_last0 >> 1) & 1);
        if (bx_last1 >= 0) tc::mbar_wait(&s_bar[1], (uint32_t)(bx_last1 >> 1) & 1);
    }
    cp_async_wait<0>();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, PL::TALLOC);
    }
}

}  // namespace rverom
