// rom_tc_wide.cuh -- tensor-core evaluation kernel for wide planar ROMs
// (augmented size NA = n~ + 4 of 36 or 68: up to 32 or 64 modes); steps
// a1-a5 of Sec. 3.2 with the contraction of Eqs. ROMintforce, ROMstiffness
// (the augmented system of Eq. Biot_Tangent) on tcgen05.
//
// Same roles, arithmetic and workspace records as eval_tc_ws_kernel
// (rom_tc_ws.cuh): tile warps evaluate the law (double-float), build their
// tile's A rows and issue its three TF32 MMA passes per k-step; helper warps
// (one or two per TMEM lane quarter) fold the TMEM accumulators (Kahan),
// tile by tile, releasing each tile warp as its tile is done, accumulate the
// float64-accurate residual and homogenized stress, stage the tables and
// write the records.
// What changes with the width:
//  - A-operand rows are the modes only (NAR = n~max rows per point: 32 or
//    64, so 4 or 2 points per 128-row tile).  The MMA yields K and K_qF
//    (columns n..n+3 of [B_i | I] are the identity); the K_FF block,
//    sum_i w_i A_i, is summed on the CUDA cores (warp shuffles per chunk,
//    double-float over chunks) and written into the record by the tile
//    warps.
//  - N = 48 or 80 columns: an accumulator and its running sum take 2N TMEM
//    columns per tile, so NW = 512 / 2N tile warps (5 or 3).
//  - The accumulators are folded every FK k-steps (a fold group; 3 FK MMAs
//    per fold) instead of once per chunk: the accumulation error of the wide
//    systems needs a fold every 4 (32 modes) or 2 (64 modes) k-steps for the
//    1e-8 stress gate.  Barriers chunk[w] and fold[w] then advance once per
//    fold group.
//  - No register reallocation: with 288 or 352 threads every warp has the
//    registers it needs at launch.
// Hand-offs (mbarriers, every wait bounded by tc::WAIT_LIMIT_NS; after the
// first timeout of a CTA no wait blocks, nothing more is issued, the tile's
// points are marked ST_TIMEOUT, and the end-of-kernel drain waits for the
// MMAs and copies in flight before TMEM is freed):
//   staged[b]  tables of a chunk in buffer b landed (cp.async arrivals)
//   bx[b]      B-operand image of a chunk in buffer b landed (bulk copy)
//   commit[w]  MMAs of tile warp w (per A buffer) completed
//   chunk[w]   MMAs of a fold group of tile warp w completed
//   wp[b]      w_i P_i of a chunk written by every tile warp (buffer b)
//   res[b]     residual of the chunk in buffer b done (w P buffer free)
//   fold[w]    accumulators of tile w's last fold group folded (free again)
//   drain      every MMA of every tile warp completed (before TMEM is freed)
#pragma once

#include "rom_tc.cuh"

namespace rverom {

template <int D, int NA, int CI, int FK>
struct TcWidePlan {
    static constexpr int G = D * D;
    static constexpr int NS = Dims<D>::NS;
    static constexpr int NQ = NA - G;
    static constexpr int QP = NQ | 1;
    static constexpr int BP = NQ | 1;
    static constexpr int NAR = NQ;                  // A-operand rows per point (the modes)
    static constexpr int JN = NAR / 32;             // rows of a point per lane and k-row group
    static constexpr int PPT = 128 / NAR;           // points per 128-row tile
    static constexpr int NN = (NA + 15) / 16 * 16;  // MMA N (columns of Bext)
    static constexpr int NW = 512 / (2 * NN);       // tile warps = tiles
    static constexpr int NH = NN > 64 ? 8 : 4;      // helper warps (NH / 4 per TMEM lane quarter)
    static constexpr int NT = 32 * (NW + NH);
    static constexpr int NHT = 32 * NH;             // helper threads
    static constexpr int NP = NW * PPT;             // points per CTA tile
    static constexpr int EPS = 8 / G;               // ECM points per k-step of 8
    static constexpr int KSC = CI / EPS;            // k-steps per chunk
    static constexpr int NGR = KSC / FK;            // fold groups per chunk
    static constexpr int RPH = (NP * NQ + NHT - 1) / NHT;  // residual rows per helper thread
    static constexpr int TCOLS = 2 * NW * NN;       // accumulator + running sum
    static constexpr int TALLOC = TCOLS <= 256 ? 256 : 512;
    static constexpr int SOFF = TALLOC / 2;         // first column of the running sums
    static constexpr int NKF = G * (G + 1) / 2;     // K_FF entries (symmetric)
    static_assert(D == 2, "planar RVEs (two ECM points per k-step)");
    static_assert(NAR == 32 || NAR == 64, "32 or 64 mode rows per point");
    static_assert(CI * PPT == 32, "one law evaluation per lane and chunk");
    static_assert(CI % EPS == 0 && KSC % FK == 0, "a chunk holds whole fold groups");
    static_assert(FK >= 2, "a group's first two k-steps are issued together");
    static_assert(NN % 16 == 0 && NW >= 1, "fold in blocks of 16 columns");
    static_assert(NP * G <= NHT, "one homogenized-stress entry per helper thread");
    static_assert(TCOLS <= 512, "TMEM holds 512 columns");
    static_assert(NW * NN <= SOFF, "accumulators, then running sums from column SOFF");
    // byte offsets
    static constexpr size_t YWARP = 4 * 4096;  // per tile warp: [2 buffers][hi|lo][2 kg][16 rg][8][4] floats
    static constexpr size_t o_Y = 0;
    static constexpr size_t BXPART = (size_t)NN * 32;
    static constexpr size_t BXBUF = (size_t)KSC * 2 * BXPART;
    static constexpr size_t o_BX = tc_al(o_Y + NW * YWARP);
    static constexpr size_t NBST = (size_t)CI * G * BP;  // (hi, lo) pairs per staging buffer
    static constexpr size_t o_B = tc_al(o_BX + 2 * BXBUF);
    static constexpr size_t o_w = tc_al(o_B + 2 * NBST * 8);
    static constexpr size_t o_ph = tc_al(o_w + 2 * 2 * CI * 4);
    static constexpr size_t o_W = tc_al(o_ph + 2 * CI * 4);                  // [warp][il][p][G*G]
    static constexpr size_t WPBUF = (size_t)NP * CI * G;                     // (hi, lo) pairs per buffer
    static constexpr size_t o_WP = tc_al(o_W + (size_t)NP * CI * G * G * 4);  // [2][warp][il][c][p]
    static constexpr size_t o_q = tc_al(o_WP + 2 * WPBUF * 8);
    static constexpr size_t o_q64 = tc_al(o_q + (size_t)NP * QP * 8);
    static constexpr size_t o_U = tc_al(o_q64 + (size_t)NP * QP * 8);
    static constexpr size_t o_R = tc_al(o_U + (size_t)NP * G * 8);
    static constexpr size_t o_dU = tc_al(o_R + (size_t)NP * G * 8);
    static constexpr size_t o_Udf = tc_al(o_dU + (size_t)NP * NS * 8);
    static constexpr size_t o_flag = tc_al(o_Udf + 2 * (size_t)NP * G * 4);
    static constexpr size_t o_pidx = o_flag + NP * 4;
    // mbarriers: bx[2], commit[NW][2], staged[2], wp[2], res[2], fold[NW], chunk[NW], drain
    static constexpr int NBAR = 2 + 2 * NW + 2 + 2 + 2 + NW + NW + 1;
    static constexpr size_t o_bar = tc_al(o_pidx + NP * 4);
    static constexpr size_t o_slot = o_bar + NBAR * 8;
    static constexpr size_t bytes = tc_al(o_slot + 8);
    static_assert(bytes <= 227 * 1024, "shared memory");
};

template <int D, int NA, int CI, int FK>
__global__ void __launch_bounds__(TcWidePlan<D, NA, CI, FK>::NT, 1) eval_tc_wide_kernel(EvalArgs a) {
    using PL = TcWidePlan<D, NA, CI, FK>;
    constexpr int G = PL::G, NS = PL::NS, NQ = PL::NQ, QP = PL::QP, BP = PL::BP, NP = PL::NP;
    constexpr int NAR = PL::NAR, JN = PL::JN, PPT = PL::PPT, NN = PL::NN, NW = PL::NW, NH = PL::NH;
    constexpr int EPS = PL::EPS, KSC = PL::KSC, NGR = PL::NGR, NT = PL::NT, NHT = PL::NHT, RPH = PL::RPH;
    constexpr int NBST = (int)PL::NBST, WPBUF = (int)PL::WPBUF, NKF = PL::NKF;
    using CR = CondRec<D, NA>;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_BX = reinterpret_cast<float *>(smem + PL::o_BX);
    float2 *s_Bst = reinterpret_cast<float2 *>(smem + PL::o_B);  // (hi, lo) of the B table: [buf][il * G + c][BP]
    float *s_wst = reinterpret_cast<float *>(smem + PL::o_w);
    int *s_ph = reinterpret_cast<int *>(smem + PL::o_ph);
    float *s_W = reinterpret_cast<float *>(smem + PL::o_W);
    float2 *s_WP = reinterpret_cast<float2 *>(smem + PL::o_WP);  // (hi, lo) of w_i P_i
    float2 *s_q2 = reinterpret_cast<float2 *>(smem + PL::o_q);    // (hi, lo) of q: [p][QP]
    double *s_qd = reinterpret_cast<double *>(smem + PL::o_q64);
    double *s_U = reinterpret_cast<double *>(smem + PL::o_U);
    double *s_R = reinterpret_cast<double *>(smem + PL::o_R);
    double *s_dU = reinterpret_cast<double *>(smem + PL::o_dU);
    float *s_Uh = reinterpret_cast<float *>(smem + PL::o_Udf), *s_Ul = s_Uh + NP * G;
    int *s_flag = reinterpret_cast<int *>(smem + PL::o_flag);
    int *s_pidx = reinterpret_cast<int *>(smem + PL::o_pidx);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem + PL::o_bar);
    uint64_t *b_bx = s_bar, *b_commit = s_bar + 2, *b_staged = b_commit + 2 * NW;
    uint64_t *b_wp = b_staged + 2, *b_res = b_wp + 2, *b_fold = b_res + 2, *b_chunk = b_fold + NW;
    uint64_t *b_drain = b_chunk + NW;
    uint32_t *s_slot = reinterpret_cast<uint32_t *>(smem + PL::o_slot);
    volatile int *s_err = reinterpret_cast<volatile int *>(smem + PL::o_slot + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool helper = warp >= NW;
    const int n = a.t.n, m = a.t.m;
    const int64_t count = a.count ? (int64_t)(*a.count) : a.n_points;
    const int64_t off = (a.perm && a.offset) ? (int64_t)(*a.offset) : 0;
    const int32_t *perm = a.perm ? a.perm + off : nullptr;
    float *ws = a.cond + off * CR::W;  // records of this type's points, by list position
    // this CTA's share of the list: a contiguous range (shares differ by at
    // most one point), taken in tiles of NP points with a partial last tile
    const int64_t r_begin = count * blockIdx.x / gridDim.x, r_end = count * (blockIdx.x + 1) / gridDim.x;
    const int nch = (m + CI - 1) / CI;

    if (warp == 0) {
        tc::tmem_alloc(s_slot, PL::TALLOC);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2 + 2 * NW; ++b) tc::mbar_init(&s_bar[b], 1);
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&b_staged[b], NHT);
            tc::mbar_init(&b_wp[b], NW);
            tc::mbar_init(&b_res[b], NH);
        }
        for (int w = 0; w < NW; ++w) {
            tc::mbar_init(&b_fold[w], NH);
            tc::mbar_init(&b_chunk[w], 1);
        }
        tc::mbar_init(b_drain, NW);
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
    // bounded wait; after the first timeout no wait blocks any more
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*s_err == 0 && !tc::mbar_wait(bar, parity)) *s_err = 1;
    };
    // helper threads: tables of chunk ch (CTA-wide chunk index g) into buffer g & 1
    int64_t bx_last0 = -1, bx_last1 = -1;  // last chunk index g bulk-copied into each buffer (issuing thread)
    auto stage = [&](uint32_t g, int ch) {
        if (*s_err != 0) return;
        const int b = g & 1, i0s = ch * CI, ht = tid - NW * 32;
        float *b2 = reinterpret_cast<float *>(s_Bst + b * NBST);
        float *wh = s_wst + b * 2 * CI, *wl = wh + CI;
        const int cnt = min(CI, m - i0s) * G * n;
        for (int x = ht; x < cnt; x += NHT) {
            const int r = x / n, j = x - r * n;  // r = il * G + c
            const int64_t gi = (int64_t)i0s * G * n + x;
            cp_async4(b2 + 2 * (r * BP + j), a.t.Bh + gi);
            cp_async4(b2 + 2 * (r * BP + j) + 1, a.t.Bl + gi);
        }
        if (ht < min(CI, m - i0s)) {
            cp_async4(wh + ht, a.t.wh + i0s + ht);
            cp_async4(wl + ht, a.t.wl + i0s + ht);
            cp_async4(s_ph + b * CI + ht, a.t.phase + i0s + ht);
        }
        tc::cp_async_mbar_arrive(&b_staged[b]);
        if (ht == 0) {
            if (b) bx_last1 = g; else bx_last0 = g;
            tc::mbar_arrive_expect_tx(&b_bx[b], (uint32_t)PL::BXBUF);
            tc::bulk_g2s(s_BX + b * (PL::BXBUF / 4), a.t.Bimg + (size_t)ch * (PL::BXBUF / 4), (uint32_t)PL::BXBUF,
                         &b_bx[b]);
        }
    };

    const uint32_t tbase = *s_slot;
    // the CTA-wide barriers (id 0) of the two roles pair up: A after the
    // polar split and micro update, B after the chunks, C after the records
    if (helper) {
        // ===================== helper warps =====================================
        uint32_t gc = 0, gg = 0;  // chunks and fold groups of this CTA before the current tile
        for (int64_t t0 = r_begin; t0 < r_end; t0 += NP) {
            const int nlive = (int)min((int64_t)NP, r_end - t0);  // points of this tile
            stage(gc, 0);
            if (nch > 1) stage(gc + 1, 1);
            tc::named_bar(0, NT);  // A
            dacc rdacc[2 * RPH];
            df pudf{0.0f, 0.0f};
            const int ht = tid - NW * 32, qd = warp & 3, hh = (warp - NW) >> 2;
            const uint32_t lanes = (uint32_t)(qd * 32) << 16;
            // residual rows o = ht + NHT u: point o / NQ, mode o % NQ
            int bo[RPH], wo[RPH];
#pragma unroll
            for (int u = 0; u < RPH; ++u) {
                const int o = ht + NHT * u;
                const bool in = o < NP * NQ;
                const int p = in ? o / NQ : 0;
                bo[u] = in ? o % NQ : 0;
                wo[u] = (p / PPT) * CI * G * PPT + p % PPT;  // w P of point p: [warp][il][c][pl]
            }
#pragma unroll
            for (int u = 0; u < 2 * RPH; ++u) rdacc[u] = dacc{0.0f, 0.0f};
            const int pp = ht / G, pc = ht % G;  // homogenized-stress entry of this thread
            const int pwo = (pp / PPT) * CI * G * PPT + pp % PPT;

            for (int ch = 0; ch < nch; ++ch) {
                const uint32_t g = gc + ch;
                const int b = g & 1;
                // folds of the chunk's groups, tile by tile: wait for the group's
                // last commit of the tile warp, fold lane quarter qd of its tile,
                // Kahan-compensated (the negated compensation goes into the
                // accumulator, onto which the next group's MMAs add), release the
                // tile warp; the last fold of the tile writes the augmented
                // systems to the workspace
                for (int gi = 0; gi < NGR; ++gi) {
                    const uint32_t gr = gg + (uint32_t)(ch * NGR + gi);  // CTA-wide fold group
                    const bool last = (ch == nch - 1) && (gi == NGR - 1);
                    const bool kahan = ch * NGR + gi > 0;
                    int fb = 0;  // fold blocks of this group so far
                    for (int t = 0; t < NW; ++t) {
                        // one phase per group; tile warp t cannot commit group
                        // gr + 1 before this fold released its accumulators, so
                        // phase gr is the barrier's current phase or the one before
                        wait(&b_chunk[t], gr & 1);
                        __syncwarp();
                        tc::fence_after_sync();
                        // tiles without points: their rows are never read, but the
                        // tile warp's barriers advance all the same
                        if (t * PPT >= nlive) {
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(&b_fold[t]);
                            continue;
                        }
                        const int row = t * 128 + qd * 32 + lane;
                        const int p = row / NAR, jr = row % NAR;
                        // blocks of 16 columns of the accumulator and its running
                        // sum (SOFF columns further on)
                        auto fold_block = [&](int c0) {
                            constexpr int W = 16;
                            // the lane quarter's helper warps take its blocks in turn
                            if constexpr (NH > 4) {
                                if (fb++ % (NH / 4) != hh) return;
                            }
                            const uint32_t ca = tbase + lanes + t * NN + c0;
                            float va[W], vs[W];
                            tc::tmem_ld16(ca, va);
                            if (kahan) tc::tmem_ld16(ca + PL::SOFF, vs);
                            tc::tmem_wait_ld();
                            if (kahan) {
#pragma unroll
                                for (int c = 0; c < W; ++c) {
                                    const float tt = __fadd_rn(vs[c], va[c]);
                                    vs[c] = __fsub_rn(va[c], __fsub_rn(tt, vs[c]));  // -(compensation)
                                    va[c] = tt;
                                }
                                if (!last) tc::tmem_st16(ca, vs);
                            }
                            if (!last) {
                                tc::tmem_st16(ca + PL::SOFF, va);
                            } else if (jr < n && p < nlive) {
                                // lane jr holds column jr of M: entries (col, jr), col >= jr
                                // (K and K_qF; K_FF comes from the tile warps)
                                float *rm = ws + (t0 + p) * CR::W + CR::o_M;
#pragma unroll
                                for (int c = 0; c < W; ++c) {
                                    const int col = c0 + c;
                                    if (col < NA && col >= jr) rm[tri(col, jr)] = va[c];
                                }
                            }
                        };
#pragma unroll
                        for (int cb = 0; cb < NN / 16; ++cb) fold_block(cb * 16);
                        if (!last) tc::tmem_wait_st();
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&b_fold[t]);
                    }
                }
                // a4: residual and homogenized stress of chunk ch (double-float)
                wait(&b_wp[b], (g >> 1) & 1);
                wait(&b_staged[b], (g >> 1) & 1);
                {
                    const float2 *B2 = s_Bst + b * NBST;
                    const float2 *WP = s_WP + b * WPBUF;
#pragma unroll 1
                    for (int il = 0; il < CI; il += 2)
#pragma unroll
                        for (int c = 0; c < G; ++c)
#pragma unroll
                            for (int u = 0; u < RPH; ++u) {
                                const int b0 = (il * G + c) * BP + bo[u], w0 = (il * G + c) * PPT + wo[u];
                                const int b1 = b0 + G * BP, w1 = w0 + G * PPT;
                                const float2 x0 = B2[b0], y0 = WP[w0], x1 = B2[b1], y1 = WP[w1];
                                dacc_fma(rdacc[2 * u], x0.x, x0.y, y0.x, y0.y);
                                dacc_fma(rdacc[2 * u + 1], x1.x, x1.y, y1.x, y1.y);
                            }
                    if (ht < NP * G && pp < nlive) {
                        for (int il = 0; il < CI; ++il) {
                            const float2 v = WP[(il * G + pc) * PPT + pwo];
                            pudf = df_add(pudf, df{v.x, v.y});
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&b_res[b]);
                // refill buffer b with chunk ch + 2 once every helper warp is
                // done with chunk ch (the tile warps are: their commits came in)
                if (ch + 2 < nch) {
                    tc::named_bar(1, NHT);
                    stage(g + 2, ch + 2);
                }
            }
            tc::named_bar(0, NT);  // B: every warp done with the tile's chunks (flags final)
            // ---- workspace records (steps a6, a7 follow in condense_kernel):
            // residual and V0 Pbar_U (double-float), q, R, U, status
            const int err = *s_err;
#pragma unroll
            for (int u = 0; u < RPH; ++u) {
                const int o = ht + NHT * u;
                if (o < NP * NQ) {
                    const int p = o / NQ, jj = o % NQ;
                    const int64_t li = t0 + p;
                    if (p < nlive) {
                        const df v = jj < n ? df_add(dacc_get(rdacc[2 * u]), dacc_get(rdacc[2 * u + 1])) : df{0.0f, 0.0f};
                        float *rec = ws + li * CR::W;
                        rec[CR::o_rh + jj] = v.hi;
                        rec[CR::o_rl + jj] = v.lo;
                        reinterpret_cast<double *>(rec + CR::o_q)[jj] = s_qd[p * QP + jj];
                    }
                }
            }
            if (ht < NP * G) {
                const int64_t li = t0 + pp;
                if (pp < nlive) {
                    float *rec = ws + li * CR::W;
                    rec[CR::o_ph + pc] = pudf.hi;
                    rec[CR::o_pl + pc] = pudf.lo;
                    reinterpret_cast<double *>(rec + CR::o_R)[pc] = s_R[pp * G + pc];
                    reinterpret_cast<double *>(rec + CR::o_U)[pc] = s_U[pp * G + pc];
                    if (pc == 0) *reinterpret_cast<int *>(rec + CR::o_flag) = err ? ST_TIMEOUT : s_flag[pp];
                }
            }
            gc += (uint32_t)nch;
            gg += (uint32_t)(nch * NGR);
            tc::named_bar(0, NT);  // C: records written before the next tile's a1
        }
        // drain: this thread's copies (normally all consumed already)
        tc::cp_async_wait_all();
        if (tid == NW * 32) {
            if (bx_last0 >= 0) tc::mbar_wait(&b_bx[0], (uint32_t)(bx_last0 >> 1) & 1);
            if (bx_last1 >= 0) tc::mbar_wait(&b_bx[1], (uint32_t)(bx_last1 >> 1) & 1);
        }
    } else {
        // ===================== tile warps =======================================
        constexpr int NTT = 32 * NW;
        uint32_t gc = 0, gstep = 0, gg = 0;
        for (int64_t t0 = r_begin; t0 < r_end; t0 += NP) {
            const int nlive = (int)min((int64_t)NP, r_end - t0);  // points of this tile
            // ---- a1: polar split, micro update ------------------------------
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
            tc::named_bar(2, NTT);
            for (int x = tid; x < NP * NQ; x += NTT) {
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
            tc::named_bar(0, NT);  // A
            const int p0 = warp * PPT;
            const bool wlive = p0 < nlive;  // this warp's tile holds points
            float *yw = reinterpret_cast<float *>(smem + PL::o_Y + warp * PL::YWARP);
            float *Ww = s_W + warp * CI * PPT * G * G;
            uint64_t *mbar = b_commit + 2 * warp;
            const uint32_t idesc = tc::idesc_tf32(128, NN);
            const df dmu0 = df_from(a.t.mu[0]), dmu1 = df_from(a.t.mu[1]);
            const df dlam0 = df_from(a.t.kappa[0] - (2.0 / 3.0) * a.t.mu[0]);
            const df dlam1 = df_from(a.t.kappa[1] - (2.0 / 3.0) * a.t.mu[1]);
            const float kmu0 = (float)a.t.mu[0], kmu1 = (float)a.t.mu[1];
            const float klam0 = (float)(a.t.kappa[0] - (2.0 / 3.0) * a.t.mu[0]);
            const float klam1 = (float)(a.t.kappa[1] - (2.0 / 3.0) * a.t.mu[1]);
            // K_FF = sum_i w_i A_i of point p0 + lane (lanes < PPT), double-float
            df kff[NKF];
#pragma unroll
            for (int e = 0; e < NKF; ++e) kff[e] = df{0.0f, 0.0f};

            for (int ch = 0; ch < nch; ++ch) {
                const uint32_t g = gc + ch;
                const int b = g & 1;
                const int i0 = ch * CI;
                wait(&b_staged[b], (g >> 1) & 1);
                // w P buffer b was last read by the residual of chunk g - 2
                if (g >= 2) wait(&b_res[b], ((g >> 1) & 1) ^ 1);
                const float2 *B2 = s_Bst + b * NBST;
                const float *wh = s_wst + b * 2 * CI, *wl = wh + CI;
                float2 *WP2 = s_WP + b * WPBUF + warp * CI * G * PPT;

                // pointwise (this warp's points, one ECM point per lane):
                // F_i, law, w P_i (double-float), W_i = w_i A_i (float32)
                {
                    const int pl = lane % PPT, il = lane / PPT;
                    const int p = p0 + pl;
                    bool live = (s_flag[p] == ST_OK) && (i0 + il < m);
                    const int ph = s_ph[b * CI + il];
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
                    float wa[G * G];
                    if (live) {
                        const float muk = ph ? kmu1 : kmu0, lam = ph ? klam1 : klam0;
                        const float c3 = muk - lam * lnJk;
                        const float wk = wh[il];
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            float Ar[G];
                            nh_tangent_row<D, float>(fi, lam, c3, muk, c, Ar);
#pragma unroll
                            for (int e = 0; e < G; ++e) wa[c * G + e] = wk * Ar[e];
                            Wt[c] = make_float4(wa[c * G], wa[c * G + 1], wa[c * G + 2], wa[c * G + 3]);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            WP2[(il * G + c) * PPT + pl] = make_float2(0.0f, 0.0f);
                            Wt[c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        }
#pragma unroll
                        for (int e = 0; e < G * G; ++e) wa[e] = 0.0f;
                    }
                    // K_FF: sum over the chunk's ECM points (lanes of equal pl),
                    // then into the double-float total of lane pl
                    int e = 0;
#pragma unroll
                    for (int c = 0; c < G; ++c)
#pragma unroll
                        for (int d2 = c; d2 < G; ++d2, ++e) {
                            float v = wa[c * G + d2];
#pragma unroll
                            for (int o = PPT; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                            kff[e] = df_add_f(kff[e], v);
                        }
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&b_wp[b]);

                // a5: per k-step, this warp builds its tile's A rows (the mode
                // rows j < n of Y_i = w_i A_i [B_i | I]) and issues its three MMAs
                for (int ks = 0; ks < KSC; ++ks) {
                    const uint32_t s = gstep + (uint32_t)(ch * KSC + ks);
                    const int gl = ch * NGR + ks / FK;           // fold group within the tile
                    const uint32_t gr = gg + (uint32_t)gl;       // CTA-wide fold group
                    const int yb = s & 1;
                    if (s >= 2) wait(&mbar[yb], ((s - 2) >> 1) & 1);
                    float *Yh = yw + yb * 2048, *Yl = Yh + 1024;
#pragma unroll
                    for (int e = 0; e < EPS; ++e) {
                        if (!wlive) break;
                        const int il = ks * EPS + e;
                        float bx[JN][G];
#pragma unroll
                        for (int h = 0; h < JN; ++h) {
                            const int j = h * 32 + lane;
#pragma unroll
                            for (int d = 0; d < G; ++d) bx[h][d] = (j < n) ? B2[(il * G + d) * BP + j].x : 0.0f;
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int rl = k * 32 + lane;  // row within the tile
                            const int pl = rl / NAR, h = (rl % NAR) / 32;
                            const float4 *Wt = reinterpret_cast<const float4 *>(Ww + (il * PPT + pl) * G * G);
                            float y[G];
#pragma unroll
                            for (int c = 0; c < G; ++c) {
                                const float4 wv = Wt[c];
                                float v = wv.x * bx[h][0];
                                v = __fmaf_rn(wv.y, bx[h][1], v);
                                v = __fmaf_rn(wv.z, bx[h][2], v);
                                v = __fmaf_rn(wv.w, bx[h][3], v);
                                y[c] = v;
                            }
                            float hi[G], lo[G];
#pragma unroll
                            for (int c = 0; c < G; ++c) tc::split_tf32(y[c], hi[c], lo[c]);
                            const int off2 = e * 512 + rl * 4;
                            *reinterpret_cast<float4 *>(Yh + off2) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                            *reinterpret_cast<float4 *>(Yl + off2) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                        }
                    }
                    tc::fence_proxy_async();
                    __syncwarp();
                    // the first k-step of a fold group is issued together with
                    // the second: both A buffers are built (the second needs
                    // only the MMAs of the previous group's last k-step) while
                    // the helpers still fold the previous group
                    const int kg = ks % FK;
                    if (kg == 0) continue;
                    if (lane == 0) {
                        if (ks == 1) wait(&b_bx[b], (g >> 1) & 1);
                        // the accumulators of the previous fold group were folded
                        if (kg == 1 && gr >= 1) wait(&b_fold[warp], (gr - 1) & 1);
                    }
                    if (lane == 0 && *s_err == 0) {
                        tc::fence_after_sync();
                        const uint32_t dt = tbase + warp * NN;
#pragma unroll
                        for (int q2 = (kg == 1 ? 1 : 0); q2 >= 0; --q2) {
                            // k-step ks - q2 of this chunk (k-step s - q2 of the CTA)
                            const int ki = ks - q2;
                            const int ybi = (int)((s - q2) & 1);
                            const float *Yhi = yw + ybi * 2048, *Ylo = Yhi + 1024;
                            const uint32_t ba = tc::smem_u32(s_BX + b * (PL::BXBUF / 4) + ki * 2 * (PL::BXPART / 4));
                            const uint64_t bdh = tc::smem_desc(ba, 128, 256);
                            const uint64_t bdl = tc::smem_desc(ba + (uint32_t)PL::BXPART, 128, 256);
                            const uint64_t adh = tc::smem_desc(tc::smem_u32(Yhi), 2048, 128);
                            const uint64_t adl = tc::smem_desc(tc::smem_u32(Ylo), 2048, 128);
                            // a group's first MMA starts the accumulator fresh in the
                            // first two groups of a tile; later it adds onto the
                            // fold's compensation term
                            tc::mma_tf32(dt, adh, bdh, idesc, (ki % FK > 0 || gl >= 2) ? 1u : 0u);
                            tc::mma_tf32(dt, adh, bdl, idesc, 1u);
                            tc::mma_tf32(dt, adl, bdh, idesc, 1u);
                            tc::mma_commit(&mbar[ybi]);
                        }
                        if (kg == FK - 1) tc::mma_commit(&b_chunk[warp]);  // the whole fold group
                    }
                    __syncwarp();
                }
            }
            // K_FF of this warp's points into their records (the helpers'
            // last fold writes the other entries of M)
            if (lane < PPT && p0 + lane < nlive) {
                float *rm = ws + (t0 + p0 + lane) * CR::W + CR::o_M;
                int e = 0;
#pragma unroll
                for (int c = 0; c < G; ++c)
#pragma unroll
                    for (int d2 = c; d2 < G; ++d2, ++e) rm[tri(n + d2, n + c)] = kff[e].hi + kff[e].lo;
            }
            tc::named_bar(0, NT);  // B
            gc += (uint32_t)nch;
            gstep += (uint32_t)(nch * KSC);
            gg += (uint32_t)(nch * NGR);
            tc::named_bar(0, NT);  // C
        }
        // drain: the completion of every MMA this warp issued (immediate
        // unless a timeout skipped the fold waits), before TMEM is freed
        if (lane == 0) {
            tc::mma_commit(b_drain);
            tc::mbar_wait(b_drain, 0);
        }
        __syncwarp();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, PL::TALLOC);
    }
}

}  // namespace rverom
