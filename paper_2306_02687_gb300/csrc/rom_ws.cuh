// rom_ws.cuh -- warp-specialized kernel of the mixed-precision evaluation.
//
// Same computation as eval_kernel<..., float, false> (steps a1-a7), organised
// so that the two halves of the ECM loop overlap on every SM sub-partition:
//
//   producer warps (NPW = NP * CI threads, one (point, ECM point) task each)
//     stage the chunk of the gradient table, evaluate F_i = U + B_i q and the
//     law in double-float, write w_i P_i and Y_i = w_i A_i [B_i | I] (float32)
//     into stage s of a two-stage shared-memory ring, then accumulate the
//     double-float reduced residual r and homogenized stress of the chunk;
//   consumer warps (NG = NP * tiles threads) hold register tiles of the
//     augmented system M = sum_i [B_i | I]^T Y_i, contract stage s and fold
//     the chunk partial into a Kahan-compensated sum.
//
// Hand-off uses named barriers (bar.sync / bar.arrive with a thread count):
//   FULL[s]  producers arrive after writing stage s, consumers sync on it;
//   EMPTY[s] consumers arrive after contracting stage s only when a later
//            chunk (kc + 2) will reuse it, producers sync on it before
//            restaging (kc >= 2), so arrivals and waits pair exactly;
//   PBAR     producer-only barrier (staged table visible, w P complete);
//   GBAR     consumer-only barrier before the accumulators are spilled.
// Every thread runs the same tile and chunk loops (uniform trip counts), so
// each barrier generation completes.
#pragma once
#include "rom_core.cuh"

namespace rverom {

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int D, int NA, int TA, int TB, int NP, int CI>
struct WsPlan {
    static constexpr int G = D * D;
    static constexpr int NS = Dims<D>::NS;
    static constexpr int NQ = NA - G;
    static constexpr int QP = NQ | 1;
    static constexpr int BP = NQ | 1;
    static constexpr int NAP = NA + 1;
    static constexpr int TPP = (NA / TA) * (NA / TB);
    static constexpr int NG = NP * TPP;   // consumer threads
    static constexpr int NPW = NP * CI;   // producer threads
    static constexpr int NT = NPW + NG;
    static constexpr int KC = CI * G;
    static constexpr int NRI = 2 * NP * NA;  // items (point, row j of [r; V0 Pbar_U], component half)
    static constexpr int RPT = (NRI + NPW - 1) / NPW;
    static_assert(NA % TA == 0 && NA % TB == 0, "tile must divide NA");
    static_assert(NG % 32 == 0 && NPW % 32 == 0 && NT <= 1024, "roles must be whole warps");
    static_assert(NP * NA * NA <= 2 * NP * KC * NAP, "accumulator spill must fit in the ring");
    // floats
    static constexpr int f_Y = 0;                         // [2][KC][NP][NAP]
    static constexpr int f_Bx = f_Y + 2 * NP * KC * NAP;  // [2][KC][NA]
    static constexpr int f_Bh = f_Bx + 2 * KC * NA;       // [2][CI*G][BP]
    static constexpr int f_Bl = f_Bh + 2 * CI * G * BP;
    static constexpr int f_wh = f_Bl + 2 * CI * G * BP;   // [2][CI]
    static constexpr int f_wl = f_wh + 2 * CI;
    static constexpr int f_WPh = f_wl + 2 * CI;           // [CI*G][NP]
    static constexpr int f_WPl = f_WPh + CI * G * NP;
    static constexpr int f_qh = f_WPl + CI * G * NP;      // [NP][QP]
    static constexpr int f_ql = f_qh + NP * QP;
    static constexpr int f_Uh = f_ql + NP * QP;           // [NP][G]
    static constexpr int f_Ul = f_Uh + NP * G;
    static constexpr int f_X = f_Ul + NP * G;             // [NP][G][NQ]
    static constexpr int f_rp = f_X + NP * G * NQ;        // residual halves as double-float [2][NRI]
    static constexpr int n_f = ((f_rp + 2 * NRI + 1) / 2) * 2;
    // doubles
    static constexpr int d_qd = 0;
    static constexpr int d_U = d_qd + NP * QP;
    static constexpr int d_R = d_U + NP * G;
    static constexpr int d_dU = d_R + NP * G;
    static constexpr int d_r = d_dU + NP * NS;
    static constexpr int d_PU = d_r + NP * NQ;
    static constexpr int d_y = d_PU + NP * G;
    static constexpr int n_d = d_y + NP * NA;
    // ints
    static constexpr int i_ph = 0;                        // [2][CI]
    static constexpr int i_flag = i_ph + 2 * CI;
    static constexpr int i_pidx = i_flag + NP;
    static constexpr int n_i = i_pidx + NP;
    static constexpr size_t bytes = 8 * (size_t)n_d + 4 * (size_t)n_f + 4 * (size_t)n_i;
};

template <int D, int NA, int TA, int TB, int NP, int CI>
__global__ void __launch_bounds__(WsPlan<D, NA, TA, TB, NP, CI>::NT, 1) eval_ws_kernel(EvalArgs a) {
    using PL = WsPlan<D, NA, TA, TB, NP, CI>;
    constexpr int G = PL::G, NS = PL::NS, NQ = PL::NQ, QP = PL::QP, BP = PL::BP, NAP = PL::NAP;
    constexpr int TPP = PL::TPP, NG = PL::NG, NPW = PL::NPW, NT = PL::NT, KC = PL::KC, RPT = PL::RPT;
    constexpr int NRI = PL::NRI;
    constexpr int NTB = NA / TB;
    constexpr int B_FULL = 1, B_EMPTY = 3, B_P = 5, B_G = 6;
    extern __shared__ __align__(16) unsigned char smem[];
    double *sd = reinterpret_cast<double *>(smem);
    float *sf = reinterpret_cast<float *>(sd + PL::n_d);
    int *si = reinterpret_cast<int *>(sf + PL::n_f);
    double *s_qd = sd + PL::d_qd, *s_U = sd + PL::d_U, *s_R = sd + PL::d_R, *s_dU = sd + PL::d_dU;
    double *s_r = sd + PL::d_r, *s_PU = sd + PL::d_PU, *s_y = sd + PL::d_y;
    float *s_Y = sf + PL::f_Y, *s_Bx = sf + PL::f_Bx, *s_Bh = sf + PL::f_Bh, *s_Bl = sf + PL::f_Bl;
    float *s_wh = sf + PL::f_wh, *s_wl = sf + PL::f_wl, *s_WPh = sf + PL::f_WPh, *s_WPl = sf + PL::f_WPl;
    float *s_qh = sf + PL::f_qh, *s_ql = sf + PL::f_ql, *s_Uh = sf + PL::f_Uh, *s_Ul = sf + PL::f_Ul;
    float *s_X = sf + PL::f_X, *s_rp = sf + PL::f_rp;
    float *s_M = s_Y;
    int *s_ph = si + PL::i_ph, *s_flag = si + PL::i_flag, *s_pidx = si + PL::i_pidx;

    const int tid = threadIdx.x;
    const bool producer = tid < NPW;
    const int n = a.t.n, m = a.t.m;
    const int nch = (m + CI - 1) / CI;
    const int64_t count = a.count ? (int64_t)(*a.count) : a.n_points;
    const int32_t *perm = a.perm ? a.perm + (a.offset ? *a.offset : 0) : nullptr;
    const int64_t n_tiles = (count + NP - 1) / NP;
    const df dmu0 = df_from(a.t.mu[0]), dmu1 = df_from(a.t.mu[1]);
    const df dlam0 = df_from(a.t.kappa[0] - (2.0 / 3.0) * a.t.mu[0]);
    const df dlam1 = df_from(a.t.kappa[1] - (2.0 / 3.0) * a.t.mu[1]);
    const float kmu0 = (float)a.t.mu[0], kmu1 = (float)a.t.mu[1];
    const float klam0 = dlam0.hi, klam1 = dlam1.hi;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---- a1: polar split and micro update (all threads) -----------------
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
            const df v2 = df_from(qv);
            s_qh[p * QP + j] = v2.hi;
            s_ql[p * QP + j] = v2.lo;
        }
        __syncthreads();

        if (producer) {
            // ================= producer warps ==================================
            const int pt = tid;
            dacc rd[RPT];
#pragma unroll
            for (int u = 0; u < RPT; ++u) rd[u] = dacc{0.0f, 0.0f};
            for (int kc = 0; kc < nch; ++kc) {
                const int s = kc & 1;
                const int i0 = kc * CI;
                if (kc >= 2) named_sync(B_EMPTY + s, NT);
                float *Bh = s_Bh + s * CI * G * BP, *Bl = s_Bl + s * CI * G * BP;
                float *Bx = s_Bx + s * KC * NA;
                for (int x = pt; x < CI * G * NQ; x += NPW) {
                    const int il = x / (G * NQ), rem = x % (G * NQ), c = rem / NQ, j = rem % NQ;
                    const bool in = i0 + il < m && j < n;
                    const int64_t gi = ((int64_t)(i0 + il) * G + c) * n + j;
                    Bh[(il * G + c) * BP + j] = in ? a.t.Bh[gi] : 0.0f;
                    Bl[(il * G + c) * BP + j] = in ? a.t.Bl[gi] : 0.0f;
                }
                for (int x = pt; x < KC * NA; x += NPW) {
                    const int k = x / NA, col = x % NA, il = k / G, c = k % G;
                    float v = 0.0f;
                    if (i0 + il < m) {
                        if (col < n) v = a.t.Bh[((int64_t)(i0 + il) * G + c) * n + col];
                        else if (col - n == c) v = 1.0f;
                    }
                    Bx[x] = v;
                }
                if (pt < CI) {
                    const bool ok = i0 + pt < m;
                    const df w2 = df_from(ok ? a.t.w[i0 + pt] : 0.0);
                    s_wh[s * CI + pt] = w2.hi;
                    s_wl[s * CI + pt] = w2.lo;
                    s_ph[s * CI + pt] = ok ? a.t.phase[i0 + pt] : 0;
                }
                named_sync(B_P, NPW);

                // pointwise task (p, il): F_i, law, w P_i, Y_i
                {
                    const int p = pt % NP, il = pt / NP;
                    float *Ys = s_Y + s * NP * KC * NAP;
                    float *yrow = Ys + ((il * G) * NP + p) * NAP;
                    bool live = (s_flag[p] == ST_OK) && (i0 + il < m);
                    const int ph = s_ph[s * CI + il];
                    float fi[G], lnf = 0.0f;
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
                        if (!nh_stress_df<D>(F, ph ? dmu1 : dmu0, ph ? dlam1 : dlam0, P, fi, lnf)) {
                            atomicCAS(&s_flag[p], ST_OK, ST_DETF);
                            live = false;
                        } else {
                            const df w2{s_wh[s * CI + il], s_wl[s * CI + il]};
#pragma unroll
                            for (int c = 0; c < G; ++c) {
                                const df wp = df_mul(w2, P[c]);
                                s_WPh[(il * G + c) * NP + p] = wp.hi;
                                s_WPl[(il * G + c) * NP + p] = wp.lo;
                            }
                        }
                    }
                    if (live) {
                        const float muk = ph ? kmu1 : kmu0, lam = ph ? klam1 : klam0;
                        const float c3 = muk - lam * lnf;
                        const float *bx = Bx + il * G * NA;
                        const float wk = s_wh[s * CI + il];
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            float Ar[G];
                            nh_tangent_row<D, float>(fi, lam, c3, muk, c, Ar);
                            float *yr = yrow + c * NP * NAP;
                            // [B_i | I | 0] row block: the identity columns give w A_i
#pragma unroll
                            for (int b = 0; b < NA; ++b) {
                                float v = 0.0f;
#pragma unroll
                                for (int c2 = 0; c2 < G; ++c2) v = kfma(Ar[c2], bx[c2 * NA + b], v);
                                yr[b] = wk * v;
                            }
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            s_WPh[(il * G + c) * NP + p] = 0.0f;
                            s_WPl[(il * G + c) * NP + p] = 0.0f;
                            float *yr = yrow + c * NP * NAP;
                            for (int b = 0; b < NA; ++b) yr[b] = 0.0f;
                        }
                    }
                }
                named_sync(B_P, NPW);
                named_arrive(B_FULL + s, NT);

                // double-float residual rows j < n and homogenized-stress rows
                // j = n + c (identity modes) of the chunk; each item owns one
                // half of the chunk's ECM points, items interleaved for ILP
                for (int il = 0; il < CI; ++il) {
#pragma unroll
                    for (int cc = 0; cc < G / 2 + (G & 1); ++cc) {
#pragma unroll
                        for (int u = 0; u < RPT; ++u) {
                            const int item = pt + u * NPW;
                            const int c = 2 * cc + (item & 1);  // component half of the item
                            if (item < NRI && c < G) {
                                const int o = item >> 1;
                                const int p = o / NA, j = o % NA;
                                const int wi = (il * G + c) * NP + p;
                                if (j < n) {
                                    const int bi = (il * G + c) * BP + j;
                                    dacc_fma(rd[u], Bh[bi], Bl[bi], s_WPh[wi], s_WPl[wi]);
                                } else if (j - n == c) {
                                    dacc_fma(rd[u], 1.0f, 0.0f, s_WPh[wi], s_WPl[wi]);
                                }
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int item = pt + u * NPW;
                if (item < NRI) {
                    const df v = dacc_get(rd[u]);
                    s_rp[2 * item] = v.hi;
                    s_rp[2 * item + 1] = v.lo;
                }
            }
        } else {
            // ================= consumer warps ==================================
            const int gt = tid - NPW;
            const int tp = gt / TPP, tt = gt % TPP;
            const int a0 = (tt / NTB) * TA, b0 = (tt % NTB) * TB;
            float acc[TA][TB], kh[TA][TB], kc2[TA][TB];
#pragma unroll
            for (int x = 0; x < TA; ++x)
#pragma unroll
                for (int y = 0; y < TB; ++y) {
                    acc[x][y] = 0.0f;
                    kh[x][y] = 0.0f;
                    kc2[x][y] = 0.0f;
                }
            for (int kc = 0; kc < nch; ++kc) {
                const int s = kc & 1;
                named_sync(B_FULL + s, NT);
                const float *Bx = s_Bx + s * KC * NA;
                const float *Yp = s_Y + s * NP * KC * NAP + tp * NAP + b0;
#pragma unroll 4
                for (int k = 0; k < KC; ++k) {
                    float av[TA], bv[TB];
#pragma unroll
                    for (int x = 0; x < TA; ++x) av[x] = Bx[k * NA + a0 + x];
#pragma unroll
                    for (int y = 0; y < TB; ++y) bv[y] = Yp[k * NP * NAP + y];
#pragma unroll
                    for (int x = 0; x < TA; ++x)
#pragma unroll
                        for (int y = 0; y < TB; ++y) acc[x][y] = __fmaf_rn(av[x], bv[y], acc[x][y]);
                }
                if (kc + 2 < nch) named_arrive(B_EMPTY + s, NT);
#pragma unroll
                for (int x = 0; x < TA; ++x)
#pragma unroll
                    for (int y = 0; y < TB; ++y) {
                        const float yv = __fsub_rn(acc[x][y], kc2[x][y]);
                        const float t = __fadd_rn(kh[x][y], yv);
                        kc2[x][y] = __fsub_rn(__fsub_rn(t, kh[x][y]), yv);
                        kh[x][y] = t;
                        acc[x][y] = 0.0f;
                    }
            }
            named_sync(B_G, NG);
#pragma unroll
            for (int x = 0; x < TA; ++x)
#pragma unroll
                for (int y = 0; y < TB; ++y) s_M[(tp * NA + a0 + x) * NA + b0 + y] = kh[x][y] - kc2[x][y];
        }
        __syncthreads();
        // combine the two halves of every row
        for (int o = tid; o < NP * NA; o += NT) {
            const int p = o / NA, j = o % NA;
            const df h0{s_rp[4 * o], s_rp[4 * o + 1]}, h1{s_rp[4 * o + 2], s_rp[4 * o + 3]};
            const double v = df_to(df_add(h0, h1));
            if (j < NQ) s_r[p * NQ + j] = v;
            if (j >= n && j < n + G) s_PU[p * G + j - n] = v;
        }
        __syncthreads();

        // ---- a6: condensation, one warp per point -------------------------
        const int warp = tid >> 5, lane = tid & 31;
        for (int p = warp; p < NP; p += NT / 32) {
            if (s_flag[p] != ST_OK) continue;
            const int st = condense_warp<D, NA, NQ, float, float>(s_M + p * NA * NA, s_y + p * NA,
                                                                 s_X + p * G * NQ, s_r + p * NQ, s_PU + p * G,
                                                                 n, lane);
            if (lane == 0 && st != ST_OK) s_flag[p] = st;
        }
        __syncthreads();
        // ---- a7: outputs ---------------------------------------------------
        for (int p = warp; p < NP; p += NT / 32) {
            const int gp = s_pidx[p];
            if (gp < 0) continue;
            write_outputs_warp<D, NA, NQ, float, float>(a, gp, s_flag[p], n, s_y + p * NA, s_X + p * G * NQ,
                                                      s_M + p * NA * NA, s_qd + p * QP, s_r + p * NQ,
                                                      s_R + p * G, s_U + p * G, lane);
        }
        __syncthreads();
    }
}

}  // namespace rverom
