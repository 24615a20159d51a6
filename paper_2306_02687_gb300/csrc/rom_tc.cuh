// rom_tc.cuh -- mixed-precision evaluation kernel whose reduced-tangent
// contraction (step a5, Eqs. ROMstiffness and Biot_Tangent of Sec. 3.2) runs
// on the tcgen05 tensor cores.
//
// The augmented system of one macro point alpha,
//     M_alpha = sum_i Bext_i^T Y_i,  Y_i = w_i A_i Bext_i,  Bext_i = [B_i | I],
// is computed for all points of a CTA at once as one matrix product whose
// shared operand is the gradient table:
//     D[(alpha, j), c] = sum_k Y[k, (alpha, j)] Bext[k, c],   k = (i, component)
// A operand: the Y rows of the CTA's points stacked along M (NAR rows per
//            point, 128-row MMA tiles), built in shared memory per k-step.
// B operand: Bext, pre-split on the host into TF32 leading and trailing parts
//            and pre-arranged in the MMA's core-matrix layout, so that a chunk
//            of ECM points is one contiguous bulk (TMA) copy.
// Precision: three TF32 products per k-step (Yhi Bhi + Yhi Blo + Ylo Bhi)
// give float32-level products; the float32 accumulator in TMEM is started
// fresh every chunk of CI ECM points and added into a running sum (also in
// TMEM), which bounds the accumulation error like the compensated chunk sums
// of the SIMT kernel.
// Everything else (a1-a4, a6, a7) is the mixed form of the SIMT kernel:
// double-float kinematics, law, residual and homogenized stress; float32
// tangent and factorization; register-resident condensation.
#pragma once

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
    static constexpr int NAR = (NA + 7) / 8 * 8;    // A-operand rows per point
    static constexpr int NN = (NA + 15) / 16 * 16;  // MMA N (columns of Bext)
    static constexpr int ROWS = NP * NAR;
    static constexpr int MT = (ROWS + 127) / 128;   // 128-row MMA tiles
    static constexpr int MROWS = MT * 128;
    static constexpr int EPS = 8 / G;               // ECM points per k-step of 8
    static constexpr int KSC = CI / EPS;            // k-steps per chunk
    static constexpr int NT = 256;
    static constexpr int RPT = (NP * NQ + NT - 1) / NT;
    // chunks per fold group: the tensor core's float32 accumulation does not
    // round to nearest (it behaves like truncation), so its accumulator is
    // restarted every chunk (at most 3 * KSC MMAs) and the chunk results are
    // added, rounded to nearest, into the running sum
    static constexpr int FG = 1;
    static constexpr int TCOLS = 2 * MT * NN;       // accumulator + running sum
    static constexpr int TALLOC = TCOLS <= 32 ? 32 : TCOLS <= 64 ? 64 : TCOLS <= 128 ? 128 : TCOLS <= 256 ? 256 : 512;
    static_assert(D == 2, "planar RVEs (one or two ECM points per k-step)");
    static_assert(CI % EPS == 0, "a chunk holds whole k-steps");
    static_assert(TCOLS <= 512, "TMEM holds 512 columns");
    static_assert(NA <= 32, "register-resident condensation");
    static_assert(NP * CI >= NT / 2, "law phase keeps most threads busy");
    // byte offsets
    static constexpr size_t YPART = (size_t)MT * 4096;  // one k-step, one part (hi or lo)
    static constexpr size_t MBYTES = (size_t)NP * NA * NA * 4;
    static constexpr size_t o_Y = 0;  // [2 buffers][hi|lo][MT][2 kg][16 rg][8][4]; later M[NP][NA][NA]
    static constexpr size_t BXPART = (size_t)NN * 32;    // [NN/8][2 kg][8][4] floats
    static constexpr size_t BXBUF = (size_t)KSC * 2 * BXPART;
    static constexpr size_t o_BX = tc_al(o_Y + (4 * YPART > MBYTES ? 4 * YPART : MBYTES));
    static constexpr size_t NBST = (size_t)CI * G * BP;  // floats per part of a staging buffer
    static constexpr size_t o_B = tc_al(o_BX + 2 * BXBUF);
    static constexpr size_t o_w = tc_al(o_B + 2 * 2 * NBST * 4);
    static constexpr size_t o_ph = tc_al(o_w + 2 * 2 * CI * 4);
    static constexpr size_t o_W = tc_al(o_ph + 2 * CI * 4);
    static constexpr size_t o_WP = tc_al(o_W + (size_t)CI * NP * G * G * 4);
    static constexpr size_t o_q = tc_al(o_WP + 2 * (size_t)CI * G * NP * 4);
    static constexpr size_t o_q64 = tc_al(o_q + 2 * (size_t)NP * QP * 4);
    static constexpr size_t o_U = tc_al(o_q64 + (size_t)NP * QP * 8);
    static constexpr size_t o_R = tc_al(o_U + (size_t)NP * G * 8);
    static constexpr size_t o_dU = tc_al(o_R + (size_t)NP * G * 8);
    static constexpr size_t o_Udf = tc_al(o_dU + (size_t)NP * NS * 8);
    static constexpr size_t o_r = tc_al(o_Udf + 2 * (size_t)NP * G * 4);
    static constexpr size_t o_PU = tc_al(o_r + 2 * (size_t)NP * NQ * 4);
    static constexpr size_t o_flag = tc_al(o_PU + 2 * (size_t)NP * G * 4);
    static constexpr size_t o_pidx = o_flag + NP * 4;
    static constexpr size_t o_bar = tc_al(o_pidx + NP * 4);  // 4 mbarriers, TMEM slot, error flag
    static constexpr size_t bytes = o_bar + 64;
    static_assert(bytes <= 227 * 1024, "shared memory");
};

// Image of Bext for the B operand: per k-step of 8 (k = i * G + c), the TF32
// leading part then the trailing part, each [nn/8][2][8][4] floats.
// Defined with the host-side table preparation.
template <int D, int NA, int NP, int CI>
__global__ void __launch_bounds__(256, 1) eval_tc_kernel(EvalArgs a) {
    using PL = TcPlan<D, NA, NP, CI>;
    constexpr int G = PL::G, NS = PL::NS, NQ = PL::NQ, QP = PL::QP, BP = PL::BP;
    constexpr int NAR = PL::NAR, NN = PL::NN, MT = PL::MT, MROWS = PL::MROWS;
    constexpr int EPS = PL::EPS, KSC = PL::KSC, NT = PL::NT, RPT = PL::RPT;
    constexpr int NBST = (int)PL::NBST;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *s_Y = reinterpret_cast<float *>(smem + PL::o_Y);
    float *s_Mf = reinterpret_cast<float *>(smem + PL::o_Y);
    float *s_BX = reinterpret_cast<float *>(smem + PL::o_BX);
    float *s_Bst = reinterpret_cast<float *>(smem + PL::o_B);
    float *s_wst = reinterpret_cast<float *>(smem + PL::o_w);
    int *s_ph = reinterpret_cast<int *>(smem + PL::o_ph);
    float *s_W = reinterpret_cast<float *>(smem + PL::o_W);
    float *s_WPh = reinterpret_cast<float *>(smem + PL::o_WP), *s_WPl = s_WPh + CI * G * NP;
    float *s_qh = reinterpret_cast<float *>(smem + PL::o_q), *s_ql = s_qh + NP * QP;
    double *s_qd = reinterpret_cast<double *>(smem + PL::o_q64);
    double *s_U = reinterpret_cast<double *>(smem + PL::o_U);
    double *s_R = reinterpret_cast<double *>(smem + PL::o_R);
    double *s_dU = reinterpret_cast<double *>(smem + PL::o_dU);
    float *s_Uh = reinterpret_cast<float *>(smem + PL::o_Udf), *s_Ul = s_Uh + NP * G;
    float *s_rh = reinterpret_cast<float *>(smem + PL::o_r), *s_rl = s_rh + NP * NQ;
    float *s_puh = reinterpret_cast<float *>(smem + PL::o_PU), *s_pul = s_puh + NP * G;
    int *s_flag = reinterpret_cast<int *>(smem + PL::o_flag);
    int *s_pidx = reinterpret_cast<int *>(smem + PL::o_pidx);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + PL::o_bar);  // [0,1] table copies, [2,3] MMA commits
    uint32_t *s_slot = reinterpret_cast<uint32_t *>(smem + PL::o_bar + 32);
    int *s_err = reinterpret_cast<int *>(smem + PL::o_bar + 36);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.t.n, m = a.t.m;
    const int na = n + G;
    const int64_t count = a.count ? (int64_t)(*a.count) : a.n_points;
    const int32_t *perm = a.perm ? a.perm + (a.offset ? *a.offset : 0) : nullptr;
    const int64_t n_tiles = (count + NP - 1) / NP;
    const int nch = (m + CI - 1) / CI;

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
        for (int b = 0; b < 4; ++b) tc::mbar_init(&s_bar[b], 1);
        tc::mbar_init_fence();
        *s_err = 0;
    }
    // staging buffers: zero once (entries past m keep finite values)
    for (int x = tid; x < 2 * 2 * NBST; x += NT) s_Bst[x] = 0.0f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *s_slot;
    const uint32_t idesc = tc::idesc_tf32(128, NN);
    uint32_t gstep = 0, gchunk = 0;  // k-steps and chunks issued by this CTA so far

    auto stage_cp = [&](int buf, int i0s) {
        float *bh = s_Bst + buf * 2 * NBST, *bl = bh + NBST;
        float *wh = s_wst + buf * 2 * CI, *wl = wh + CI;
        const int cnt = min(CI, m - i0s) * G * n;
        for (int x = tid; x < cnt; x += NT) {
            const int r = x / n, j = x - r * n;  // r = il * G + c
            const int64_t gi = (int64_t)i0s * G * n + x;
            cp_async4(bh + r * BP + j, a.t.Bh + gi);
            cp_async4(bl + r * BP + j, a.t.Bl + gi);
        }
        if (tid < min(CI, m - i0s)) {
            cp_async4(wh + tid, a.t.wh + i0s + tid);
            cp_async4(wl + tid, a.t.wl + i0s + tid);
            cp_async4(s_ph + buf * CI + tid, a.t.phase + i0s + tid);
        }
        cp_async_commit();
    };
    auto stage_bulk = [&](int buf, int ch) {  // one thread
        tc::mbar_arrive_expect_tx(&s_bar[buf], (uint32_t)PL::BXBUF);
        tc::bulk_g2s(s_BX + buf * (PL::BXBUF / 4), a.t.Bimg + (size_t)ch * (PL::BXBUF / 4), (uint32_t)PL::BXBUF,
                     &s_bar[buf]);
    };

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---- a1: polar split, micro update ---------------------------------
        if (tid < NP) {
            const int p = tid;
            const int64_t li = tile * NP + p;
            int gp = -1;
            if (li < count) gp = perm ? perm[li] : (int)li;
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
            s_qh[p * QP + j] = v.hi;
            s_ql[p * QP + j] = v.lo;
        }
        dacc rdacc[2 * RPT];
#pragma unroll
        for (int u = 0; u < 2 * RPT; ++u) rdacc[u] = dacc{0.0f, 0.0f};
        df pudf{0.0f, 0.0f};
        __syncthreads();

        // ---- ECM loop: a2-a5 ----------------------------------------------
        stage_cp(gchunk & 1, 0);
        if (tid == 0) stage_bulk(gchunk & 1, 0);
        bool fresh = true;  // the next MMA starts a fold group
        int folds = 0;
        for (int ch = 0; ch < nch; ++ch, ++gchunk) {
            const int buf = gchunk & 1;
            const int i0 = ch * CI;
            if (ch + 1 < nch) {
                stage_cp(buf ^ 1, i0 + CI);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float *Bh = s_Bst + buf * 2 * NBST, *Bl = Bh + NBST;
            const float *wh = s_wst + buf * 2 * CI, *wl = wh + CI;

            // pointwise: F_i, law, w P_i (double-float), W_i = w_i A_i (float32)
            for (int task = tid; task < NP * CI; task += NT) {
                const int p = task % NP, il = task / NP;
                bool live = (s_flag[p] == ST_OK) && (i0 + il < m);
                const int ph = s_ph[buf * CI + il];
                float fi[G];
                float lnJk = 0.0f;
                if (live) {
                    df F[G], P[G];
                    const float *bh = Bh + il * G * BP, *bl = Bl + il * G * BP;
                    const float *qh = s_qh + p * QP, *ql = s_ql + p * QP;
                    dacc sacc[G];
#pragma unroll
                    for (int c = 0; c < G; ++c) sacc[c] = dacc{s_Uh[p * G + c], s_Ul[p * G + c]};
                    for (int j = 0; j < n; ++j) {
                        const float qhj = qh[j], qlj = ql[j];
#pragma unroll
                        for (int c = 0; c < G; ++c) dacc_fma(sacc[c], bh[c * BP + j], bl[c * BP + j], qhj, qlj);
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
                            s_WPh[(il * G + c) * NP + p] = wp.hi;
                            s_WPl[(il * G + c) * NP + p] = wp.lo;
                        }
                    }
                }
                float *Wt = s_W + (il * NP + p) * G * G;
                if (live) {
                    const float muk = ph ? kmu1 : kmu0, lam = ph ? klam1 : klam0;
                    const float c3 = muk - lam * lnJk;
                    const float wk = wh[il];
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        float Ar[G];
                        nh_tangent_row<D, float>(fi, lam, c3, muk, c, Ar);
#pragma unroll
                        for (int e = 0; e < G; ++e) Wt[c * G + e] = wk * Ar[e];
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        s_WPh[(il * G + c) * NP + p] = 0.0f;
                        s_WPl[(il * G + c) * NP + p] = 0.0f;
                    }
#pragma unroll
                    for (int e = 0; e < G * G; ++e) Wt[e] = 0.0f;
                }
            }
            __syncthreads();
            // next chunk's table image; its buffer was last read by the MMAs of chunk ch-1
            if (tid == 0 && ch + 1 < nch) {
                if (ch > 0 && !tc::mbar_wait(&s_bar[2 + ((gstep - 1) & 1)], ((gstep - 1) >> 1) & 1)) *s_err = 1;
                stage_bulk(buf ^ 1, ch + 1);
            }

            // a5: per k-step, build Y (A operand) and issue the MMAs
            for (int ks = 0; ks < KSC; ++ks) {
                const uint32_t s = gstep + ks;
                const int yb = s & 1;
                if (s >= 2 && !tc::mbar_wait(&s_bar[2 + yb], ((s - 2) >> 1) & 1)) *s_err = 1;
                float *Yh = s_Y + yb * 2 * (PL::YPART / 4), *Yl = Yh + PL::YPART / 4;
                for (int task = tid; task < EPS * MROWS; task += NT) {
                    const int r = task % MROWS, e = task / MROWS;
                    const int il = ks * EPS + e;
                    const int p = r / NAR, j = r - p * NAR;
                    float y[G];
#pragma unroll
                    for (int c = 0; c < G; ++c) y[c] = 0.0f;
                    if (p < NP && j < na) {
                        const float *Wt = s_W + (il * NP + p) * G * G;
                        float bx[G];
#pragma unroll
                        for (int d = 0; d < G; ++d) bx[d] = (j < n) ? Bh[(il * G + d) * BP + j] : ((j - n == d) ? 1.0f : 0.0f);
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            float v = 0.0f;
#pragma unroll
                            for (int d = 0; d < G; ++d) v = __fmaf_rn(Wt[c * G + d], bx[d], v);
                            y[c] = v;
                        }
                    }
                    float hi[G], lo[G];
#pragma unroll
                    for (int c = 0; c < G; ++c) tc::split_tf32(y[c], hi[c], lo[c]);
                    const int off = (r >> 7) * 1024 + e * 512 + (r & 127) * 4;
                    *reinterpret_cast<float4 *>(Yh + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<float4 *>(Yl + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                }
                tc::fence_proxy_async();
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after_sync();
                    if (ks == 0 && !tc::mbar_wait(&s_bar[buf], (gchunk >> 1) & 1)) *s_err = 1;
                    const uint32_t ya = tc::smem_u32(Yh), yla = tc::smem_u32(Yl);
                    const uint32_t ba = tc::smem_u32(s_BX + buf * (PL::BXBUF / 4) + ks * 2 * (PL::BXPART / 4));
                    const uint64_t bdh = tc::smem_desc(ba, 128, 256);
                    const uint64_t bdl = tc::smem_desc(ba + (uint32_t)PL::BXPART, 128, 256);
#pragma unroll 1
                    for (int t = 0; t < MT; ++t) {
                        const uint32_t dt = tbase + t * NN;
                        const uint64_t adh = tc::smem_desc(ya + t * 4096, 2048, 128);
                        const uint64_t adl = tc::smem_desc(yla + t * 4096, 2048, 128);
                        tc::mma_tf32(dt, adh, bdh, idesc, fresh ? 0u : 1u);
                        tc::mma_tf32(dt, adh, bdl, idesc, 1u);
                        tc::mma_tf32(dt, adl, bdh, idesc, 1u);
                    }
                    tc::mma_commit(&s_bar[2 + yb]);
                }
                fresh = false;
            }
            gstep += KSC;

            // a4: float64-accurate reduced residual and homogenized stress
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int o = tid + u * NT;
                if (o < NP * NQ) {
                    const int p = o / NQ, j = o % NQ;
                    if (j < n) {
                        dacc v0 = rdacc[2 * u], v1 = rdacc[2 * u + 1];
                        for (int il = 0; il < CI; il += 2)
#pragma unroll
                            for (int c = 0; c < G; ++c) {
                                const int b0 = (il * G + c) * BP + j, w0 = (il * G + c) * NP + p;
                                const int b1 = b0 + G * BP, w1 = w0 + G * NP;
                                dacc_fma(v0, Bh[b0], Bl[b0], s_WPh[w0], s_WPl[w0]);
                                dacc_fma(v1, Bh[b1], Bl[b1], s_WPh[w1], s_WPl[w1]);
                            }
                        rdacc[2 * u] = v0;
                        rdacc[2 * u + 1] = v1;
                    }
                }
            }
            if (tid < NP * G) {
                const int p = tid / G, c = tid % G;
                for (int il = 0; il < CI; ++il)
                    pudf = df_add(pudf, df{s_WPh[(il * G + c) * NP + p], s_WPl[(il * G + c) * NP + p]});
            }

            // fold the group accumulator into the running sum (TMEM); the last
            // fold writes the augmented system of every point to shared memory
            const bool last = (ch == nch - 1);
            if ((ch + 1) % PL::FG == 0 || last) {
                const uint32_t sl = gstep - 1;
                if (!tc::mbar_wait(&s_bar[2 + (sl & 1)], (sl >> 1) & 1)) *s_err = 1;
                __syncwarp();  // the TMEM loads below are warp-collective
                tc::fence_after_sync();
                const int qd = warp & 3;
                const uint32_t lanes = (uint32_t)(qd * 32) << 16;
                for (int t = warp >> 2; t < MT; t += 2) {
                    const int row = t * 128 + qd * 32 + lane;
                    const int p = row / NAR, j = row - p * NAR;
#pragma unroll
                    for (int cb = 0; cb < NN / 16; ++cb) {
                        float va[16], vs[16];
                        tc::tmem_ld16(tbase + lanes + t * NN + cb * 16, va);
                        if (folds > 0) tc::tmem_ld16(tbase + lanes + MT * NN + t * NN + cb * 16, vs);
                        tc::tmem_wait_ld();
                        if (folds > 0) {
#pragma unroll
                            for (int c = 0; c < 16; ++c) va[c] = __fadd_rn(vs[c], va[c]);
                        }
                        if (!last) {
                            tc::tmem_st16(tbase + lanes + MT * NN + t * NN + cb * 16, va);
                        } else if (p < NP && j < NA) {
#pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const int col = cb * 16 + c;
                                if (col < NA) s_Mf[(p * NA + col) * NA + j] = va[c];
                            }
                        }
                    }
                }
                if (!last) tc::tmem_wait_st();
                tc::fence_before_sync();
                fresh = true;
                ++folds;
            }
            __syncthreads();
        }

        // ---- spill the residual and Pbar_U (double-float pairs) -------------
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int o = tid + u * NT;
            if (o < NP * NQ) {
                const df v = df_add(dacc_get(rdacc[2 * u]), dacc_get(rdacc[2 * u + 1]));
                s_rh[o] = v.hi;
                s_rl[o] = v.lo;
            }
        }
        if (tid < NP * G) {
            s_puh[tid] = pudf.hi;
            s_pul[tid] = pudf.lo;
        }
        __syncthreads();
        // ---- a6, a7: condensation and outputs, one warp per point -----------
        for (int p = warp; p < NP; p += NT / 32) {
            const int gp = s_pidx[p];
            if (gp < 0) continue;
            condense_out_regs_mix<D, NA, NQ>(a, s_Mf + p * NA * NA, s_rh + p * NQ, s_rl + p * NQ, s_puh + p * G,
                                             s_pul + p * G, gp, s_flag[p], n, s_qd + p * QP, s_R + p * G,
                                             s_U + p * G, (float)(1.0 / a.V0), lane);
        }
        __syncthreads();
        if (*s_err && tid < NP && s_pidx[tid] >= 0) a.status[s_pidx[tid]] = ST_TIMEOUT;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, PL::TALLOC);
    }
}

}  // namespace rverom
