// rom_condense.cuh -- static condensation (step a6) and outputs (a7) of the
// mixed form with one thread per macro point (Sec. 3.2.3, Eq. Biot_Tangent,
// written for the first Piola-Kirchhoff stress).
//
// The tensor-core evaluation kernel leaves, per point, a workspace record
// with the augmented system M = [[K, K_qF], [K_Fq, K_FF]] (float32, lower
// triangle packed by rows), the double-float right-hand side [r; V0 Pbar_U],
// the micro-updated amplitudes q, the polar factors R, U and the status so
// far.  This kernel factors the K block of M in float32 (Cholesky, SPD for
// the hyperelastic law) carrying the coupling rows through the elimination,
// so that the trailing block becomes V0 C_U = K_FF - K_Fq K^-1 K_qF.  The
// part of the solve that reaches Pbar is carried in double-float against the
// float32 factor: w = L^-1 r and V0 Pbar_alg = V0 Pbar_U - Z w (Z = K_Fq L^-T,
// the eliminated coupling rows).  The Newton correction s = L^-T w and
// X = K^-1 K_qF (S = X E) are float32 (iterative refinement: the next
// evaluation's float64-accurate residual corrects them).  Outputs as the other kernels: P = R Pbar_alg, the consistent
// tangent through the polar derivative, the new micro state and the
// residual norm.
//
// A CTA holds CT points (the lanes of a warp) and TPP warps: warp r works on
// the rows i = r (mod TPP) of every point, lane pt on point pt.  The records'
// matrices are staged in shared memory as [entry][point] (row pitch CT + 1:
// the lanes of a warp touch consecutive banks), so every step of the
// factorization is one conflict-free shared-memory access per point; CTA
// barriers separate the column scaling and the trailing update of a pivot
// step.  Eight warps per 32 points (TPP = 8; 4 and 16 measured slower on
// the 24-mode ROM) keep several warps per scheduler busy although each
// point's matrix occupies 1.8 KB of shared memory.
#pragma once

#include "rom_core.cuh"

namespace rverom {

// workspace record of one point, in 4-byte words (float64 fields at even words)
template <int D, int NA>
struct CondRec {
    static constexpr int G = D * D;
    static constexpr int NQ = NA - G;
    static constexpr int o_q = 0;             // float64 [NQ]: q after the micro update
    static constexpr int o_R = o_q + 2 * NQ;  // float64 [G]: rotation of the polar split
    static constexpr int o_U = o_R + 2 * G;   // float64 [G]: stretch
    static constexpr int o_rh = o_U + 2 * G;  // float [NQ]: reduced residual r, leading part
    static constexpr int o_rl = o_rh + NQ;    // float [NQ]: trailing part
    static constexpr int o_ph = o_rl + NQ;    // float [G]: V0 Pbar_U, leading part
    static constexpr int o_pl = o_ph + G;     // float [G]: trailing part
    static constexpr int o_flag = o_pl + G;   // int: status after steps a1-a5
    static constexpr int o_M = (o_flag + 1 + 3) / 4 * 4;  // float [NA (NA + 1) / 2]: M, lower, by rows
    static constexpr int NL = NA * (NA + 1) / 2;
    static constexpr int W = (o_M + NL + 3) / 4 * 4;  // words per record
};
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

template <int D, int NA, int CT, int TPP>
struct CondPlan {
    static constexpr int G = D * D, NQ = NA - G, NL = CondRec<D, NA>::NL;
    static constexpr int LD = CT + 1;
    static constexpr int o_A = 0;                // [NL][LD]: M, then its factor
    static constexpr int o_Yh = o_A + NL * LD;   // [NQ][LD]: r, then w = L^-1 r (double-float)
    static constexpr int o_Yl = o_Yh + NQ * LD;
    static constexpr int o_P = o_Yl + NQ * LD;   // [2][G][LD]: V0 Pbar_alg (double-float)
    static constexpr int o_st = o_P + 2 * G * LD;  // int [LD]: status
    static constexpr size_t bytes = (size_t)(o_st + LD) * sizeof(float);
};

template <int D, int NA, int CT, int TPP>
__global__ void __launch_bounds__(CT * TPP) condense_kernel(EvalArgs a) {
    using CR = CondRec<D, NA>;
    using CP = CondPlan<D, NA, CT, TPP>;
    constexpr int G = CR::G, NQ = CR::NQ, NS = Dims<D>::NS, NL = CR::NL, W = CR::W, LD = CP::LD;
    extern __shared__ __align__(16) unsigned char smem[];
    float *sm = reinterpret_cast<float *>(smem);
    float *A = sm + CP::o_A, *Yh = sm + CP::o_Yh, *Yl = sm + CP::o_Yl;
    float *Pv = sm + CP::o_P;
    int *s_st = reinterpret_cast<int *>(sm + CP::o_st);
    const int tid = threadIdx.x;
    const int r = tid / CT, pt = tid % CT;
    const int n = a.t.n, na = n + G;
    const int64_t count = a.count ? (int64_t)(*a.count) : a.n_points;
    const int64_t off = (a.perm && a.offset) ? (int64_t)(*a.offset) : 0;
    const int32_t *perm = a.perm ? a.perm + off : nullptr;
    const float *ws = a.cond + off * W;
    const float V0inv = (float)(1.0 / a.V0);
    const double dnan = __longlong_as_double(0x7ff8000000000000ll);
    float *Ac = A + pt, *yh = Yh + pt, *yl = Yl + pt;

    for (int64_t b0 = (int64_t)blockIdx.x * CT; b0 < count; b0 += (int64_t)gridDim.x * CT) {
        const int nb = (int)((count - b0) < CT ? (count - b0) : CT);
        __syncthreads();
        // stage the packed matrices and the residuals, transposed to
        // [entry][point], with asynchronous copies (all in flight at once)
        for (int x = tid; x < nb * NL; x += CT * TPP) {
            const int q = x / NL, e = x - q * NL;
            cp_async4(A + e * LD + q, ws + (b0 + q) * W + CR::o_M + e);
        }
        for (int x = tid; x < nb * NQ; x += CT * TPP) {
            const int q = x / NQ, i = x - q * NQ;
            cp_async4(Yh + i * LD + q, ws + (b0 + q) * W + CR::o_rh + i);
            cp_async4(Yl + i * LD + q, ws + (b0 + q) * W + CR::o_rl + i);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        const bool valid = pt < nb;
        const int64_t li = b0 + pt;
        const float *rec = ws + li * W;
        float rmax = 0.0f;
        if (r == 0) {
            int st = ST_NONFINITE;
            if (valid) {
                st = *reinterpret_cast<const int *>(rec + CR::o_flag);
                bool fin = true;
                for (int i = 0; i < n; ++i) {
                    const float v = yh[i * LD];
                    fin = fin && isfinite(v) && isfinite(yl[i * LD]);
                    rmax = fmaxf(rmax, fabsf(v));
                }
                if (st == ST_OK && !fin) st = ST_NONFINITE;
            }
            s_st[pt] = valid ? st : -1;
        }
        __syncthreads();
        bool ok = s_st[pt] == ST_OK;
        // ---- forward: Cholesky of the K block carried through the coupling
        // rows, w = L^-1 r (double-float)
        for (int k = 0; k < n; ++k) {
            float lkk = 0.0f, inv = 0.0f;
            df wk{0.0f, 0.0f};
            if (ok) {
                const float d = Ac[tri(k, k) * LD];
                if (!(d > 0.0f) || !isfinite(d)) {
                    ok = false;
                    if (r == 0) s_st[pt] = ST_NONSPD;
                } else {
                    lkk = sqrtf(d);
                    inv = 1.0f / lkk;
                    wk = df_div_f(df{yh[k * LD], yl[k * LD]}, lkk, inv);
                    int i = k + 1 + ((r - (k + 1)) % TPP + TPP) % TPP;
                    for (; i < na; i += TPP) {
                        const float lik = Ac[tri(i, k) * LD] * inv;
                        Ac[tri(i, k) * LD] = lik;
                        if (i < n) {
                            const df v = df_sub(df{yh[i * LD], yl[i * LD]}, df_mul_f(wk, lik));
                            yh[i * LD] = v.hi;
                            yl[i * LD] = v.lo;
                        }
                    }
                }
            }
            __syncthreads();
            if (ok) {
                if (r == k % TPP) {
                    Ac[tri(k, k) * LD] = lkk;
                    yh[k * LD] = wk.hi;
                    yl[k * LD] = wk.lo;
                }
                int i = k + 1 + ((r - (k + 1)) % TPP + TPP) % TPP;
                for (; i < na; i += TPP) {
                    const float lik = Ac[tri(i, k) * LD];
                    float *row = Ac + tri(i, 0) * LD;
#pragma unroll 4
                    for (int j = k + 1; j <= i; ++j) row[j * LD] = __fmaf_rn(-lik, Ac[tri(j, k) * LD], row[j * LD]);
                }
            }
            __syncthreads();
        }
        // V0 Pbar_alg = V0 Pbar_U - Z w (double-float), component c by warp c mod TPP
        if (ok) {
            for (int c = r; c < G; c += TPP) {
                df z{0.0f, 0.0f};
                for (int j = 0; j < n; ++j) z = df_add(z, df_mul_f(df{yh[j * LD], yl[j * LD]}, Ac[tri(n + c, j) * LD]));
                const df P = df_sub(df{rec[CR::o_ph + c], rec[CR::o_pl + c]}, z);
                Pv[c * LD + pt] = P.hi;
                Pv[(G + c) * LD + pt] = P.lo;
            }
        }
        __syncthreads();
        // ---- backward, column-oriented (float32): s = L^-T w over w and
        // X = L^-T Z^T over the coupling rows Z.  Entry k of the solutions is
        // stored by its row's warp one step later (step k reads entry k in
        // every warp; step k - 1 touches only entries below k).
        int pk = -1;
        float ps = 0.0f, px[G];
        for (int k = n - 1; k >= 0; --k) {
            if (ok) {
                if (pk >= 0) {
                    yh[pk * LD] = ps;
#pragma unroll
                    for (int c = 0; c < G; ++c) Ac[tri(n + c, pk) * LD] = px[c];
                    pk = -1;
                }
                const float inv = 1.0f / Ac[tri(k, k) * LD];
                const float sk = yh[k * LD] * inv;
                float xk[G];
#pragma unroll
                for (int c = 0; c < G; ++c) xk[c] = Ac[tri(n + c, k) * LD] * inv;
                if (r == k % TPP) {
                    pk = k;
                    ps = sk;
#pragma unroll
                    for (int c = 0; c < G; ++c) px[c] = xk[c];
                }
                for (int j = r; j < k; j += TPP) {
                    const float lkj = Ac[tri(k, j) * LD];
                    yh[j * LD] = __fmaf_rn(-lkj, sk, yh[j * LD]);
#pragma unroll
                    for (int c = 0; c < G; ++c) Ac[tri(n + c, j) * LD] = __fmaf_rn(-lkj, xk[c], Ac[tri(n + c, j) * LD]);
                }
            }
            __syncthreads();
        }
        if (ok && pk >= 0) {  // entry 0 (its row's warp reads it below)
            yh[pk * LD] = ps;
#pragma unroll
            for (int c = 0; c < G; ++c) Ac[tri(n + c, pk) * LD] = px[c];
        }
        if (!valid) continue;
        const int gp = perm ? perm[li] : (int)li;
        if (!ok) {
            if (r == 0) {
                a.status[gp] = s_st[pt];
                a.rnorm[gp] = dnan;
                for (int c = 0; c < G; ++c) a.Pbar[(int64_t)gp * G + c] = dnan;
                for (int c = 0; c < G * G; ++c) a.dPdF[(int64_t)gp * G * G + c] = dnan;
            }
            continue;
        }
        // ---- outputs: micro state (entries j = r mod TPP, each stored by
        // this warp in the backward sweep)
        const double *qrec = reinterpret_cast<const double *>(rec + CR::o_q);
        for (int j = r; j < a.nmax; j += TPP) {
            const int64_t base = (int64_t)gp * a.nmax + j;
            const bool in = j < n;
            a.q[base] = in ? qrec[j] : 0.0;
            a.s[base] = in ? (double)yh[j * LD] : 0.0;
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                int i1, j1;
                voigt_pair(D, v, i1, j1);
                float sv = 0.0f;
                if (in) {
                    sv = Ac[tri(n + i1 * D + j1, j) * LD];
                    if (i1 != j1) sv += Ac[tri(n + j1 * D + i1, j) * LD];
                }
                a.S[base * NS + v] = (double)sv;
            }
        }
        const double *Rm = reinterpret_cast<const double *>(rec + CR::o_R);
        const double *Um = reinterpret_cast<const double *>(rec + CR::o_U);
        df Pd[G];
#pragma unroll
        for (int c = 0; c < G; ++c) Pd[c] = df{Pv[c * LD + pt], Pv[(G + c) * LD + pt]};
        if (r == 0) {
            // Pbar = R Pbar_alg / V0 in double-float; Uprev = U; residual norm
            a.rnorm[gp] = (double)rmax;
            a.status[gp] = ST_OK;
            df Rd[G];
#pragma unroll
            for (int c = 0; c < G; ++c) Rd[c] = df_from(Rm[c]);
            const df iVd = df_from(1.0 / a.V0);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int J = 0; J < D; ++J) {
                    df v{0.0f, 0.0f};
#pragma unroll
                    for (int k = 0; k < D; ++k) v = df_add(v, df_mul(Rd[i * D + k], Pd[k * D + J]));
                    a.Pbar[(int64_t)gp * G + i * D + J] = df_to(df_mul(v, iVd));
                }
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                int i1, j1;
                voigt_pair(D, v, i1, j1);
                a.Uprev[(int64_t)gp * NS + v] = Um[i1 * D + j1];
            }
        }
        // consistent tangent, column e0 = (i0, J0) by warp e0 mod TPP:
        // R (C_U dU + Om Pbar_alg)
        float R[G], U[G], Pa[G], CU[G * G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            R[c] = (float)Rm[c];
            U[c] = (float)Um[c];
            Pa[c] = Pd[c].hi * V0inv;
        }
#pragma unroll
        for (int c = 0; c < G; ++c)
#pragma unroll
            for (int e = 0; e < G; ++e) CU[c * G + e] = Ac[tri(n + (c > e ? c : e), n + (c > e ? e : c)) * LD] * V0inv;
        for (int e0 = r; e0 < G; e0 += TPP) {
            const int i0 = e0 / D, J0 = e0 % D;
            float Om[G], dU[G], T[G];
            polar_dir_f<D>(R, U, i0, J0, Om, dU);
#pragma unroll
            for (int c = 0; c < G; ++c) {
                float v = 0.0f;
#pragma unroll
                for (int e = 0; e < G; ++e) v += CU[c * G + e] * dU[e];
                T[c] = v;
            }
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int J = 0; J < D; ++J) {
                    float v = T[i * D + J];
#pragma unroll
                    for (int k = 0; k < D; ++k) v += Om[i * D + k] * Pa[k * D + J];
                    T[i * D + J] = v;
                }
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int J = 0; J < D; ++J) {
                    float v = 0.0f;
#pragma unroll
                    for (int k = 0; k < D; ++k) v += R[i * D + k] * T[k * D + J];
                    a.dPdF[((int64_t)gp * G + i * D + J) * G + e0] = (double)v;
                }
        }
    }
}

}  // namespace rverom
