// rom_core.cuh -- device building blocks of the hyper-reduced RVE evaluation
// (Lange, Huetter, Kiefer, arXiv 2306.02687, Sec. 3.2-3.3 and Sec. 4).
//
//   * compressible Neo-Hooke law P(F), A = dP/dF (the micro law of the
//     synthetic workloads; the paper leaves the hyperelastic law open)
//   * polar split F = R U (Sec. 3.2.2) and the derivative dR, dU
//   * the batched evaluation kernel template (steps a1-a7 of the header)
//
// Kernel organisation (one CTA = NP macro points of one RVE type):
//   for every chunk of CI ECM points
//     stage    B rows of the chunk -> shared memory (float64 copy for the
//              FP64-accurate kinematics, KT copy extended by the identity
//              block [B_i | I] as left operand of the contraction)
//     pointwise  one thread per (point, ECM point): F_i = U + B_i q, the law,
//              w_i P_i (float64) and Y_i = w_i A_i [B_i | I] (KT) -> shared
//     contract register-tiled  M += sum_i [B_i | I]^T Y_i, i.e. the augmented
//              reduced system [[K, K_qF], [K_Fq, K_FF]] of Eq. ROMstiffness
//              plus its macro coupling, and the float64 GEMV r += B_i^T w_i P_i
//   condense one warp per point: partial Cholesky of the K block carried
//              through the coupling block and the right-hand side [r; V0 Pbar]
//              -- the trailing g x g block becomes V0 C_U and the trailing
//              right-hand side V0 Pbar_alg (static condensation, Sec. 3.2.3)
//   output   s, S, Pbar = R Pbar_alg, dPdF through the polar derivative.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "df64.cuh"

namespace rverom {

constexpr int ST_OK = 0, ST_DETF = 1, ST_NONSPD = 2, ST_NONFINITE = 3;

__device__ __forceinline__ float kfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double kfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <int D>
struct Dims {
    static constexpr int G = D * D;
    static constexpr int NS = (D == 2) ? 3 : 6;
};

// Voigt pair v -> (i, j); order 2D (11,22,12), 3D (11,22,33,12,13,23).
__host__ __device__ inline void voigt_pair(int D, int v, int &i, int &j) {
    if (D == 2) {
        const int a[3] = {0, 1, 0}, b[3] = {0, 1, 1};
        i = a[v];
        j = b[v];
    } else {
        const int a[6] = {0, 1, 2, 0, 0, 1}, b[6] = {0, 1, 2, 1, 2, 2};
        i = a[v];
        j = b[v];
    }
}

struct TypeDev {
    int n, m;
    const double *B;   // [m][g][n]
    const float *Bh;   // [m][g][n] float32 leading part of B
    const float *Bl;   // [m][g][n] float32 remainder B - Bh
    const double *w;   // [m]
    const float *wh;   // [m] float32 leading part of w
    const float *wl;   // [m] float32 remainder w - wh
    const int *phase;  // [m]
    double mu[2], kappa[2];
    // tensor-core path (planar types with n + 4 <= 32): [B_i | I] split into
    // TF32 leading/trailing parts in the MMA operand layout, per k-step of 8
    // (k = i * 4 + c): [hi|lo][img_nn / 8][2][8][4] floats
    const float *Bimg;
    int img_nn;
};

// 4-byte asynchronous global -> shared copy (no register round trip)
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct EvalArgs {
    TypeDev t;
    int64_t n_points;
    const int32_t *perm;    // point lists of all types (bucketed) or nullptr
    const int32_t *count;   // device count of this type's list, or nullptr (= n_points)
    const int32_t *offset;  // device offset of this type's list in perm
    int nmax;
    double V0;
    const double *Fbar;
    double *q, *s, *S, *Uprev;
    double *Pbar, *dPdF, *rnorm;
    int32_t *status;
    // adjoint mode only
    const double *gP;   // [n][g] cotangent on Pbar
    double *gF;         // [n][g] cotangent on Fbar (out)
    double *partials;   // [gridDim.x][4] per-CTA sums of the moduli gradient
    // tensor-core form only: per-point workspace records, indexed by the
    // point's position in the (bucketed) batch
    float *cond;
};

// ---------------------------------------------------------------------------
// small dense helpers
template <int D>
__device__ __forceinline__ double det(const double *F) {
    if (D == 2) return F[0] * F[3] - F[1] * F[2];
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// inverse via the adjugate; returns det
template <int D>
__device__ __forceinline__ double inverse(const double *F, double *Fi) {
    double J = det<D>(F);
    double r = 1.0 / J;
    if (D == 2) {
        Fi[0] = F[3] * r;
        Fi[1] = -F[1] * r;
        Fi[2] = -F[2] * r;
        Fi[3] = F[0] * r;
    } else {
        Fi[0] = (F[4] * F[8] - F[5] * F[7]) * r;
        Fi[1] = (F[2] * F[7] - F[1] * F[8]) * r;
        Fi[2] = (F[1] * F[5] - F[2] * F[4]) * r;
        Fi[3] = (F[5] * F[6] - F[3] * F[8]) * r;
        Fi[4] = (F[0] * F[8] - F[2] * F[6]) * r;
        Fi[5] = (F[2] * F[3] - F[0] * F[5]) * r;
        Fi[6] = (F[3] * F[7] - F[4] * F[6]) * r;
        Fi[7] = (F[1] * F[6] - F[0] * F[7]) * r;
        Fi[8] = (F[0] * F[4] - F[1] * F[3]) * r;
    }
    return J;
}

// ---------------------------------------------------------------------------
// Neo-Hooke: P = mu F + (lam lnJ - mu) F^-T, lam = kappa - 2 mu / 3.
// Returns false when det F <= 0 (or not finite).
template <int D>
__device__ __forceinline__ bool nh_stress(const double *F, double mu, double kappa, double *P,
                                          double *Fi, double &lnJ) {
    constexpr int G = D * D;
    double J = inverse<D>(F, Fi);
    if (!(J > 0.0) || !isfinite(J)) return false;
    lnJ = log(J);
    double lam = kappa - (2.0 / 3.0) * mu;
    double c = lam * lnJ - mu;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) P[i * D + j] = mu * F[i * D + j] + c * Fi[j * D + i];
    (void)G;
    return true;
}

// Row c = (i, J) of A[iJ][kL] = mu d_ik d_JL + lam Fi_Ji Fi_Lk + c3 Fi_Li Fi_Jk,
// c3 = mu - lam lnJ; fi is F^-1 in KT precision.
template <int D, typename KT>
__device__ __forceinline__ void nh_tangent_row(const KT *fi, KT lam, KT c3, KT mu, int c, KT *Arow) {
    const int i = c / D, J = c % D;
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int L = 0; L < D; ++L) {
            KT v = lam * fi[J * D + i] * fi[L * D + k] + c3 * fi[L * D + i] * fi[J * D + k];
            if (i == k && J == L) v += mu;
            Arow[k * D + L] = v;
        }
}

// The same row for an index c known only at run time (one row per lane):
// the entries of F^-1 that depend on i or J are picked by selects, so that
// fi stays in registers and only the lane's own row is formed.
template <int D, typename KT>
__device__ __forceinline__ void nh_tangent_row_rt(const KT *fi, KT lam, KT c3, KT mu, int c, KT *Arow) {
    const int i = c / D, J = c % D;
    KT fLi[D], fJk[D];  // Fi_Li and Fi_Jk for L, k = 0 .. D-1
#pragma unroll
    for (int t = 0; t < D; ++t) {
        fLi[t] = fi[t * D];
        fJk[t] = fi[t];
#pragma unroll
        for (int u = 1; u < D; ++u) {
            if (i == u) fLi[t] = fi[t * D + u];
            if (J == u) fJk[t] = fi[u * D + t];
        }
    }
    KT fJi = fJk[0];  // Fi_Ji
#pragma unroll
    for (int u = 1; u < D; ++u)
        if (i == u) fJi = fJk[u];
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int L = 0; L < D; ++L) {
            KT v = lam * fJi * fi[L * D + k] + c3 * fLi[L] * fJk[k];
            if (i == k && J == L) v += mu;
            Arow[k * D + L] = v;
        }
}

// Neo-Hooke stress in double-float: P = mu F + ((lam lnJ - mu)/J) cof(F),
// F^-T = cof(F)/J.  Also returns F^-1 and ln J in float32 for the tangent.
template <int D>
__device__ __forceinline__ bool nh_stress_df(const df *F, df mu, df lam, df *P, float *fi, float &lnJf) {
    constexpr int G = D * D;
    df cof[G];
    df J;
    if (D == 2) {
        cof[0] = F[3];
        cof[1] = df_neg(F[2]);
        cof[2] = df_neg(F[1]);
        cof[3] = F[0];
        J = df_sub(df_mul(F[0], F[3]), df_mul(F[1], F[2]));
    } else {
        cof[0] = df_sub(df_mul(F[4], F[8]), df_mul(F[5], F[7]));
        cof[1] = df_sub(df_mul(F[5], F[6]), df_mul(F[3], F[8]));
        cof[2] = df_sub(df_mul(F[3], F[7]), df_mul(F[4], F[6]));
        cof[3] = df_sub(df_mul(F[2], F[7]), df_mul(F[1], F[8]));
        cof[4] = df_sub(df_mul(F[0], F[8]), df_mul(F[2], F[6]));
        cof[5] = df_sub(df_mul(F[1], F[6]), df_mul(F[0], F[7]));
        cof[6] = df_sub(df_mul(F[1], F[5]), df_mul(F[2], F[4]));
        cof[7] = df_sub(df_mul(F[2], F[3]), df_mul(F[0], F[5]));
        cof[8] = df_sub(df_mul(F[0], F[4]), df_mul(F[1], F[3]));
        J = df_add(df_add(df_mul(F[0], cof[0]), df_mul(F[1], cof[1])), df_mul(F[2], cof[2]));
    }
    if (!(J.hi > 0.0f) || !isfinite(J.hi)) return false;
    const df lnJ = df_log(J);
    const df rJ = df_div(df{1.0f, 0.0f}, J);
    const df coef = df_mul(df_sub(df_mul(lam, lnJ), mu), rJ);
#pragma unroll
    for (int c = 0; c < G; ++c) P[c] = df_add(df_mul(mu, F[c]), df_mul(coef, cof[c]));
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) fi[i * D + j] = __fmul_rn(cof[j * D + i].hi, rJ.hi);
    lnJf = lnJ.hi;
    return true;
}

// The law of nh_stress_df spread over a group of LPT lanes, lane c < G
// holding F_c: lane c forms cofactor c and stress entry P_c only; F, J and
// the cofactors reach the lanes that need them by shuffles, and every lane
// gets ln J and F^-1 (float32).  Per entry the operations and their order
// are those of nh_stress_df.  Every lane of the warp calls it (it shuffles),
// so a failed J does not return early: the result is then discarded.
template <int D, int LPT>
__device__ __forceinline__ bool nh_stress_df_split(df Fc, int c, df mu, df lam, df &Pc, float *fi, float &lnJf) {
    constexpr int G = D * D;
    static_assert(G <= LPT, "one lane per entry");
    const int cc = c < G ? c : 0;
    auto sh = [](df v, int src) {
        return df{__shfl_sync(0xffffffffu, v.hi, src, LPT), __shfl_sync(0xffffffffu, v.lo, src, LPT)};
    };
    df cof, J;
    if constexpr (D == 2) {
        const df o = sh(Fc, 3 - cc);  // cof = [F3, -F2, -F1, F0]
        cof = (cc == 0 || cc == 3) ? o : df_neg(o);
        J = df_sub(df_mul(sh(Fc, 0), sh(Fc, 3)), df_mul(sh(Fc, 1), sh(Fc, 2)));
    } else {
        // cofactor (i, j) from rows r1 < r2 != i, columns j + 1, j + 2 (mod 3),
        // swapped for the middle row so that the sign is in the product order
        const int i = cc / 3, j = cc % 3;
        const int r1 = i == 0 ? 1 : 0, r2 = i == 2 ? 1 : 2;
        int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        if (i == 1) {
            const int t = j1;
            j1 = j2;
            j2 = t;
        }
        const df fa = sh(Fc, r1 * 3 + j1), fb = sh(Fc, r2 * 3 + j2);
        const df fd = sh(Fc, r1 * 3 + j2), fe = sh(Fc, r2 * 3 + j1);
        cof = df_sub(df_mul(fa, fb), df_mul(fd, fe));
        J = df_add(df_add(df_mul(sh(Fc, 0), sh(cof, 0)), df_mul(sh(Fc, 1), sh(cof, 1))), df_mul(sh(Fc, 2), sh(cof, 2)));
    }
    const bool ok = J.hi > 0.0f && isfinite(J.hi);
    const df Js = ok ? J : df{1.0f, 0.0f};
    const df lnJ = df_log(Js);
    const df rJ = df_div(df{1.0f, 0.0f}, Js);
    const df coef = df_mul(df_sub(df_mul(lam, lnJ), mu), rJ);
    Pc = df_add(df_mul(mu, Fc), df_mul(coef, cof));
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int q = 0; q < D; ++q) fi[r * D + q] = __fmul_rn(__shfl_sync(0xffffffffu, cof.hi, q * D + r, LPT), rJ.hi);
    lnJf = lnJ.hi;
    return ok;
}

// ---------------------------------------------------------------------------
// polar decomposition F = R U.  2D: closed form; 3D: Newton iteration
// X <- (X + X^-T)/2 on the rotation (quadratically convergent, bounded).
template <int D>
__device__ bool polar(const double *F, double *R, double *U) {
    constexpr int G = D * D;
    if (D == 2) {
        double a = F[0] + F[3], b = F[2] - F[1];
        double rho = sqrt(a * a + b * b);
        if (!(rho > 0.0)) return false;
        double c = a / rho, s = b / rho;
        R[0] = c;
        R[1] = -s;
        R[2] = s;
        R[3] = c;
    } else {
        double X[G], Xi[G];
#pragma unroll
        for (int x = 0; x < G; ++x) X[x] = F[x];
        for (int it = 0; it < 60; ++it) {
            double J = inverse<3>(X, Xi);
            if (!(J > 0.0)) return false;
            double dmax = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    double nx = 0.5 * (X[i * 3 + j] + Xi[j * 3 + i]);
                    dmax = fmax(dmax, fabs(nx - X[i * 3 + j]));
                    X[i * 3 + j] = nx;
                }
            if (dmax <= 1e-16) break;
        }
#pragma unroll
        for (int x = 0; x < G; ++x) R[x] = X[x];
    }
    // U = R^T F, symmetrized
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) v += R[k * D + i] * F[k * D + j];
            U[i * D + j] = v;
        }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i + 1; j < D; ++j) {
            double v = 0.5 * (U[i * D + j] + U[j * D + i]);
            U[i * D + j] = v;
            U[j * D + i] = v;
        }
    return true;
}

// For dF = e_(i0,J0): Omega (skew, R^T dR) and dU (symmetric) of the polar
// derivative, from  Omega U + U Omega = R^T dF - dF^T R.
template <int D>
__device__ void polar_dir(const double *R, const double *U, int i0, int J0, double *Om,
                          double *dU) {
    constexpr int G = D * D;
    double X[G];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) X[a * D + b] = (b == J0) ? R[i0 * D + a] : 0.0;
    double W[G];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) W[a * D + b] = X[a * D + b] - X[b * D + a];
    if (D == 2) {
        double om = W[2] / (U[0] + U[3]);
        Om[0] = 0.0;
        Om[1] = -om;
        Om[2] = om;
        Om[3] = 0.0;
    } else {
        // (tr U I - U) omega = axial(W)
        double w0 = W[7], w1 = W[2], w2 = W[3];
        double tr = U[0] + U[4] + U[8];
        double Mx[9];
#pragma unroll
        for (int x = 0; x < 9; ++x) Mx[x] = -U[x];
        Mx[0] += tr;
        Mx[4] += tr;
        Mx[8] += tr;
        double Mi[9];
        inverse<3>(Mx, Mi);
        double o0 = Mi[0] * w0 + Mi[1] * w1 + Mi[2] * w2;
        double o1 = Mi[3] * w0 + Mi[4] * w1 + Mi[5] * w2;
        double o2 = Mi[6] * w0 + Mi[7] * w1 + Mi[8] * w2;
        Om[0] = 0.0;
        Om[1] = -o2;
        Om[2] = o1;
        Om[3] = o2;
        Om[4] = 0.0;
        Om[5] = -o0;
        Om[6] = -o1;
        Om[7] = o0;
        Om[8] = 0.0;
    }
    // dU = X - Omega U, symmetrized
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            double v = X[a * D + b];
#pragma unroll
            for (int k = 0; k < D; ++k) v -= Om[a * D + k] * U[k * D + b];
            dU[a * D + b] = v;
        }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a + 1; b < D; ++b) {
            double v = 0.5 * (dU[a * D + b] + dU[b * D + a]);
            dU[a * D + b] = v;
            dU[b * D + a] = v;
        }
}

// 1/x to float64 accuracy without a float64 divide: float32 seed refined by
// two Newton steps (r <- r (2 - x r)), each doubling the correct bits.
template <typename KT>
__device__ __forceinline__ double recip_acc(KT x) {
    double r = (double)(1.0f / (float)x);
    const double xd = (double)x;
    r = r * (2.0 - xd * r);
    r = r * (2.0 - xd * r);
    return r;
}

// Static condensation of one point by one warp (step a6): in-place partial
// Cholesky of the K block of the augmented system M = [[K, K_qF],[K_Fq, K_FF]]
// (lower triangle, KT precision) carried through the coupling rows and the
// float64 right-hand side y = [r; V0 Pbar_U]; afterwards y[0:n) = s = K^-1 r,
// y[n:n+g) = V0 Pbar_alg, the trailing block of M is V0 C_U and X = K^-1 K_qF
// (g columns of length n, pitch NQ).  Returns a status code.
template <int D, int NA, int NQ, typename KT, typename XT>
__device__ int condense_warp(KT *M, double *y, XT *X, const double *r, const double *PU, int n, int lane) {
    constexpr int G = D * D;
    const int na = n + G;
    for (int i = lane; i < na; i += 32) y[i] = (i < n) ? r[i] : PU[i - n];
    bool fin = true;
    for (int i = lane; i < n; i += 32) fin = fin && isfinite(r[i]);
    fin = __all_sync(0xffffffffu, fin);
    if (!fin) return ST_NONFINITE;
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const KT piv = M[k * NA + k];
        if (!(piv > (KT)0) || !isfinite(piv)) return ST_NONSPD;
        const KT lkk = sqrt(piv);
        const double dinv = recip_acc(lkk);
        const KT inv = (KT)dinv;
        const double yk = y[k] * dinv;
        __syncwarp();
        for (int i = k + 1 + lane; i < na; i += 32) {
            const KT lik = M[i * NA + k] * inv;
            M[i * NA + k] = lik;
            y[i] -= (double)lik * yk;
        }
        if (lane == 0) {
            M[k * NA + k] = lkk;
            y[k] = yk;
        }
        __syncwarp();
        for (int i = k + 1; i < na; ++i) {
            const KT lik = M[i * NA + k];
            for (int j = k + 1 + lane; j <= i; j += 32) M[i * NA + j] -= lik * M[j * NA + k];
        }
        __syncwarp();
    }
    // s = L^-T y[0:n)  and  X = L^-T Z^T,  Z = rows n.. of the factor
    for (int x = lane; x < G * n; x += 32) {
        const int c = x / n, j = x % n;
        X[c * NQ + j] = (XT)M[(n + c) * NA + j];
    }
    __syncwarp();
    for (int k = n - 1; k >= 0; --k) {
        const double dinv = recip_acc(M[k * NA + k]);
        const double sk = y[k] * dinv;
        XT xk[G];
        const XT xinv = (XT)dinv;
#pragma unroll
        for (int c = 0; c < G; ++c) xk[c] = X[c * NQ + k] * xinv;
        __syncwarp();
        for (int i = lane; i < k; i += 32) {
            const KT lki = M[k * NA + i];
            y[i] -= (double)lki * sk;
#pragma unroll
            for (int c = 0; c < G; ++c) X[c * NQ + i] -= (XT)lki * xk[c];
        }
        if (lane == 0) {
            y[k] = sk;
#pragma unroll
            for (int c = 0; c < G; ++c) X[c * NQ + k] = xk[c];
        }
        __syncwarp();
    }
    return ST_OK;
}

// Outputs of one point by one warp (step a7): new state q, s, S, Uprev, the
// rotated algorithmic stress Pbar = R Pbar_alg, the consistent tangent
// dPbar/dFbar through the polar derivative, rnorm and status; NaN stress and
// tangent for failed points (their state is left untouched).
template <int D, int NA, int NQ, typename KT, typename XT>
__device__ void write_outputs_warp(const EvalArgs &a, int gp, int flag, int n, const double *y, const XT *X,
                                   const KT *M, const double *qd, const double *r, const double *Rm,
                                   const double *Um, int lane) {
    constexpr int G = D * D, NS = Dims<D>::NS;
    if (flag == ST_OK) {
        for (int j = lane; j < a.nmax; j += 32) {
            const int64_t base = (int64_t)gp * a.nmax + j;
            const bool in = j < n;
            a.q[base] = in ? qd[j] : 0.0;
            a.s[base] = in ? y[j] : 0.0;
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                int i1, j1;
                voigt_pair(D, v, i1, j1);
                double sv = 0.0;
                if (in) sv = (i1 == j1) ? (double)X[(i1 * D + j1) * NQ + j]
                                        : (double)X[(i1 * D + j1) * NQ + j] + (double)X[(j1 * D + i1) * NQ + j];
                a.S[base * NS + v] = sv;
            }
        }
        double rmax = 0.0;
        for (int j = lane; j < n; j += 32) rmax = fmax(rmax, fabs(r[j]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
        if (lane == 0) {
            a.rnorm[gp] = rmax;
            a.status[gp] = ST_OK;
            const double iV = 1.0 / a.V0;
            double Pa[G], R[G], U[G], CU[G * G];
#pragma unroll
            for (int c = 0; c < G; ++c) {
                Pa[c] = y[n + c] * iV;
                R[c] = Rm[c];
                U[c] = Um[c];
            }
#pragma unroll
            for (int c = 0; c < G; ++c)
#pragma unroll
                for (int e = 0; e < G; ++e) {
                    const int hi = c > e ? c : e, lo = c > e ? e : c;
                    CU[c * G + e] = (double)M[(n + hi) * NA + n + lo] * iV;
                }
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int J = 0; J < D; ++J) {
                    double v = 0.0;
#pragma unroll
                    for (int k = 0; k < D; ++k) v += R[i * D + k] * Pa[k * D + J];
                    a.Pbar[(int64_t)gp * G + i * D + J] = v;
                }
#pragma unroll
            for (int i0 = 0; i0 < D; ++i0)
#pragma unroll
                for (int J0 = 0; J0 < D; ++J0) {
                    double Om[G], dU[G], T[G];
                    polar_dir<D>(R, U, i0, J0, Om, dU);
                    // T = Omega Pa + C_U dU
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        double v = 0.0;
#pragma unroll
                        for (int e = 0; e < G; ++e) v += CU[c * G + e] * dU[e];
                        T[c] = v;
                    }
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int J = 0; J < D; ++J) {
                            double v = T[i * D + J];
#pragma unroll
                            for (int k = 0; k < D; ++k) v += Om[i * D + k] * Pa[k * D + J];
                            T[i * D + J] = v;
                        }
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int J = 0; J < D; ++J) {
                            double v = 0.0;
#pragma unroll
                            for (int k = 0; k < D; ++k) v += R[i * D + k] * T[k * D + J];
                            a.dPdF[((int64_t)gp * G + i * D + J) * G + i0 * D + J0] = v;
                        }
                }
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                int i1, j1;
                voigt_pair(D, v, i1, j1);
                a.Uprev[(int64_t)gp * NS + v] = U[i1 * D + j1];
            }
        }
    } else if (lane == 0) {
        a.status[gp] = flag;
        a.rnorm[gp] = __longlong_as_double(0x7ff8000000000000ll);
        for (int c = 0; c < G; ++c) a.Pbar[(int64_t)gp * G + c] = __longlong_as_double(0x7ff8000000000000ll);
        for (int c = 0; c < G * G; ++c) a.dPdF[(int64_t)gp * G * G + c] = __longlong_as_double(0x7ff8000000000000ll);
    }
}

// ---- mixed form: per-point phases on the float32 pipe -----------------------
// y / d to double-float accuracy for a float divisor d with reciprocal inv:
// q1 = y.hi inv, remainder y - q1 d (exact product), q2 = remainder inv.
__device__ __forceinline__ df df_div_f(df y, float d, float inv) {
    const float q1 = __fmul_rn(y.hi, inv);
    const df r = df_sub(y, df_mul_f(df{q1, 0.0f}, d));
    return fast_two_sum(q1, __fmul_rn(r.hi, inv));
}

// Static condensation of one point by one warp, mixed form: the K block of
// M is factored in float32, the right-hand side [r; V0 Pbar_U] is carried in
// double-float (yh, yl), X = K^-1 K_qF in float32.  Same algorithm and
// outputs as condense_warp.
template <int D, int NA, int NQ>
__device__ int condense_warp_mix(float *M, float *yh, float *yl, float *X, const float *rh, const float *rl,
                                 const float *puh, const float *pul, int n, int lane) {
    constexpr int G = D * D;
    const int na = n + G;
    for (int i = lane; i < na; i += 32) {
        yh[i] = (i < n) ? rh[i] : puh[i - n];
        yl[i] = (i < n) ? rl[i] : pul[i - n];
    }
    bool fin = true;
    for (int i = lane; i < n; i += 32) fin = fin && isfinite(rh[i]) && isfinite(rl[i]);
    fin = __all_sync(0xffffffffu, fin);
    if (!fin) return ST_NONFINITE;
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const float piv = M[k * NA + k];
        if (!(piv > 0.0f) || !isfinite(piv)) return ST_NONSPD;
        const float lkk = sqrtf(piv);
        const float inv = 1.0f / lkk;
        const df yk = df_div_f(df{yh[k], yl[k]}, lkk, inv);
        __syncwarp();
        for (int i = k + 1 + lane; i < na; i += 32) {
            const float lik = M[i * NA + k] * inv;
            M[i * NA + k] = lik;
            const df v = df_sub(df{yh[i], yl[i]}, df_mul_f(yk, lik));
            yh[i] = v.hi;
            yl[i] = v.lo;
        }
        if (lane == 0) {
            M[k * NA + k] = lkk;
            yh[k] = yk.hi;
            yl[k] = yk.lo;
        }
        __syncwarp();
        for (int i = k + 1; i < na; ++i) {
            const float lik = M[i * NA + k];
            for (int j = k + 1 + lane; j <= i; j += 32) M[i * NA + j] -= lik * M[j * NA + k];
        }
        __syncwarp();
    }
    for (int x = lane; x < G * n; x += 32) {
        const int c = x / n, j = x % n;
        X[c * NQ + j] = M[(n + c) * NA + j];
    }
    __syncwarp();
    for (int k = n - 1; k >= 0; --k) {
        const float lkk = M[k * NA + k];
        const float inv = 1.0f / lkk;
        const df sk = df_div_f(df{yh[k], yl[k]}, lkk, inv);
        float xk[G];
#pragma unroll
        for (int c = 0; c < G; ++c) xk[c] = X[c * NQ + k] * inv;
        __syncwarp();
        for (int i = lane; i < k; i += 32) {
            const float lki = M[k * NA + i];
            const df v = df_sub(df{yh[i], yl[i]}, df_mul_f(sk, lki));
            yh[i] = v.hi;
            yl[i] = v.lo;
#pragma unroll
            for (int c = 0; c < G; ++c) X[c * NQ + i] -= lki * xk[c];
        }
        if (lane == 0) {
            yh[k] = sk.hi;
            yl[k] = sk.lo;
#pragma unroll
            for (int c = 0; c < G; ++c) X[c * NQ + k] = xk[c];
        }
        __syncwarp();
    }
    return ST_OK;
}

// float32 polar-derivative direction (same formulas as polar_dir)
template <int D>
__device__ void polar_dir_f(const float *R, const float *U, int i0, int J0, float *Om, float *dU) {
    constexpr int G = D * D;
    float X[G], W[G];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) X[a * D + b] = (b == J0) ? R[i0 * D + a] : 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) W[a * D + b] = X[a * D + b] - X[b * D + a];
    if (D == 2) {
        const float om = W[2] / (U[0] + U[3]);
        Om[0] = 0.0f;
        Om[1] = -om;
        Om[2] = om;
        Om[3] = 0.0f;
    } else {
        const float w0 = W[7], w1 = W[2], w2 = W[3];
        const float tr = U[0] + U[4] + U[8];
        float Mx[9], Mi[9];
#pragma unroll
        for (int x = 0; x < 9; ++x) Mx[x] = -U[x];
        Mx[0] += tr;
        Mx[4] += tr;
        Mx[8] += tr;
        const float dt = Mx[0] * (Mx[4] * Mx[8] - Mx[5] * Mx[7]) - Mx[1] * (Mx[3] * Mx[8] - Mx[5] * Mx[6]) +
                         Mx[2] * (Mx[3] * Mx[7] - Mx[4] * Mx[6]);
        const float r = 1.0f / dt;
        Mi[0] = (Mx[4] * Mx[8] - Mx[5] * Mx[7]) * r;
        Mi[1] = (Mx[2] * Mx[7] - Mx[1] * Mx[8]) * r;
        Mi[2] = (Mx[1] * Mx[5] - Mx[2] * Mx[4]) * r;
        Mi[3] = (Mx[5] * Mx[6] - Mx[3] * Mx[8]) * r;
        Mi[4] = (Mx[0] * Mx[8] - Mx[2] * Mx[6]) * r;
        Mi[5] = (Mx[2] * Mx[3] - Mx[0] * Mx[5]) * r;
        Mi[6] = (Mx[3] * Mx[7] - Mx[4] * Mx[6]) * r;
        Mi[7] = (Mx[1] * Mx[6] - Mx[0] * Mx[7]) * r;
        Mi[8] = (Mx[0] * Mx[4] - Mx[1] * Mx[3]) * r;
        const float o0 = Mi[0] * w0 + Mi[1] * w1 + Mi[2] * w2;
        const float o1 = Mi[3] * w0 + Mi[4] * w1 + Mi[5] * w2;
        const float o2 = Mi[6] * w0 + Mi[7] * w1 + Mi[8] * w2;
        Om[0] = 0.0f;
        Om[1] = -o2;
        Om[2] = o1;
        Om[3] = o2;
        Om[4] = 0.0f;
        Om[5] = -o0;
        Om[6] = -o1;
        Om[7] = o0;
        Om[8] = 0.0f;
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            float v = X[a * D + b];
#pragma unroll
            for (int k = 0; k < D; ++k) v -= Om[a * D + k] * U[k * D + b];
            dU[a * D + b] = v;
        }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a + 1; b < D; ++b) {
            const float v = 0.5f * (dU[a * D + b] + dU[b * D + a]);
            dU[a * D + b] = v;
            dU[b * D + a] = v;
        }
}

// Outputs of one point by one warp, mixed form: state and rnorm by all
// lanes, Pbar = R Pbar_alg in double-float (lane 0), tangent column e by
// lane e in float32 (the tangent is a float32 quantity of this form).
template <int D, int NA, int NQ>
__device__ void write_outputs_warp_mix(const EvalArgs &a, int gp, int flag, int n, const float *yh,
                                       const float *yl, const float *X, const float *M, const double *qd,
                                       const float *rh, const double *Rm, const double *Um, float V0inv,
                                       int lane) {
    constexpr int G = D * D, NS = Dims<D>::NS;
    if (flag != ST_OK) {
        if (lane == 0) {
            a.status[gp] = flag;
            a.rnorm[gp] = __longlong_as_double(0x7ff8000000000000ll);
        }
        for (int c = lane; c < G + G * G; c += 32) {
            if (c < G) a.Pbar[(int64_t)gp * G + c] = __longlong_as_double(0x7ff8000000000000ll);
            else a.dPdF[(int64_t)gp * G * G + c - G] = __longlong_as_double(0x7ff8000000000000ll);
        }
        return;
    }
    for (int j = lane; j < a.nmax; j += 32) {
        const int64_t base = (int64_t)gp * a.nmax + j;
        const bool in = j < n;
        a.q[base] = in ? qd[j] : 0.0;
        a.s[base] = in ? df_to(df{yh[j], yl[j]}) : 0.0;
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            int i1, j1;
            voigt_pair(D, v, i1, j1);
            float sv = 0.0f;
            if (in) sv = (i1 == j1) ? X[(i1 * D + j1) * NQ + j] : X[(i1 * D + j1) * NQ + j] + X[(j1 * D + i1) * NQ + j];
            a.S[base * NS + v] = (double)sv;
        }
    }
    float rmax = 0.0f;
    for (int j = lane; j < n; j += 32) rmax = fmaxf(rmax, fabsf(rh[j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
    float R[G], U[G], Pa[G];
#pragma unroll
    for (int c = 0; c < G; ++c) {
        R[c] = (float)Rm[c];
        U[c] = (float)Um[c];
        Pa[c] = yh[n + c] * V0inv;
    }
    if (lane == 0) {
        a.rnorm[gp] = (double)rmax;
        a.status[gp] = ST_OK;
        // Pbar = R Pbar_alg with Pbar_alg = y[n:] / V0 in double-float
        const double iV = 1.0 / a.V0;
        df Rd[G], Pd[G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            Rd[c] = df_from(Rm[c]);
            Pd[c] = df{yh[n + c], yl[n + c]};
        }
        const df iVd = df_from(iV);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int J = 0; J < D; ++J) {
                df v{0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < D; ++k) v = df_add(v, df_mul(Rd[i * D + k], Pd[k * D + J]));
                a.Pbar[(int64_t)gp * G + i * D + J] = df_to(df_mul(v, iVd));
#pragma unroll
                for (int v2 = 0; v2 < NS; ++v2) {
                    int i1, j1;
                    voigt_pair(D, v2, i1, j1);
                    if (i == 0 && J == 0) a.Uprev[(int64_t)gp * NS + v2] = Um[i1 * D + j1];
                }
            }
    }
    if (lane < G) {
        const int i0 = lane / D, J0 = lane % D;
        float Om[G], dU[G], T[G];
        polar_dir_f<D>(R, U, i0, J0, Om, dU);
#pragma unroll
        for (int c = 0; c < G; ++c) {
            float v = 0.0f;
#pragma unroll
            for (int e = 0; e < G; ++e) {
                const int hi = c > e ? c : e, lo = c > e ? e : c;
                v += M[(n + hi) * NA + n + lo] * V0inv * dU[e];
            }
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
                a.dPdF[((int64_t)gp * G + i * D + J) * G + lane] = (double)v;
            }
    }
}

// Register-resident condensation and outputs of one point by one warp, mixed
// form, for augmented size NA <= 32.  Lane j holds column j of the symmetric
// augmented matrix M (rows in registers col[0..NA)); every pivot step keeps
// the trailing block symmetric (full-square update), so the L entry a lane
// needs is its own row-k element and the row entries of the other lanes come
// by warp shuffles.  The right-hand side [r; V0 Pbar_U] is double-float, the
// coupling solve X = K^-1 K_qF float32.  Writes the same outputs as
// condense_warp_mix followed by write_outputs_warp_mix; returns the status.
template <int NA>
__device__ __forceinline__ float sel(const float (&col)[NA], int k) {
    // element k (warp-uniform, 0 <= k < NA) by a select tree on the bits of k
    float t[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) t[i] = i < NA ? col[i] : 0.0f;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool hi = (k & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) t[i] = hi ? t[i + w] : t[i];
    }
    return t[0];
}

__device__ __forceinline__ df shfl_df(df v, int src) {
    return df{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = df_add(v, df{__shfl_xor_sync(0xffffffffu, v.hi, off),
                                                           __shfl_xor_sync(0xffffffffu, v.lo, off)});
    return v;
}

template <int D, int NA, int NQ>
__device__ int condense_out_regs_mix(const EvalArgs &a, const float *Msm, const float *rh, const float *rl,
                                     const float *puh, const float *pul, int gp, int flag, int n,
                                     const double *qd, const double *Rm, const double *Um, float V0inv,
                                     int lane) {
    static_assert(NA <= 32, "one column per lane");
    constexpr int G = D * D, NS = Dims<D>::NS;
    const int na = n + G;
    const int j = lane;
    const bool colj = j < na;
    float col[NA], Lc[NA];  // column j of M / of the factor L (lane j = pivot k keeps L[:, k])
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        // lower triangle only (the contraction may skip upper blocks)
        col[i] = (colj && i < na) ? Msm[(i >= j ? i * NA + j : j * NA + i)] : 0.0f;
        Lc[i] = 0.0f;
    }
    df y{0.0f, 0.0f};
    if (j < n) y = df{rh[j], rl[j]};
    else if (colj) y = df{puh[j - n], pul[j - n]};
    const float rj = (j < n) ? rh[j] : 0.0f;
    bool fin = (j < n) ? (isfinite(rh[j]) && isfinite(rl[j])) : true;
    int st = flag;
    if (st == ST_OK && !__all_sync(0xffffffffu, fin)) st = ST_NONFINITE;
    // ---- forward: Cholesky of the K block carried through coupling and rhs
    for (int k = 0; k < n && st == ST_OK; ++k) {
        const float rowk = sel(col, k);                      // M[k][j] (= M[j][k])
        const float d = __shfl_sync(0xffffffffu, rowk, k);
        if (!(d > 0.0f) || !isfinite(d)) {
            st = ST_NONSPD;
            break;
        }
        const float lkk = sqrtf(d), inv = 1.0f / lkk;
        const float l = (j > k && colj) ? rowk * inv : 0.0f;  // L[j][k]
        const df yk = df_div_f(shfl_df(y, k), lkk, inv);
        if (j > k && colj) y = df_sub(y, df_mul_f(yk, l));
        if (j == k) y = yk;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const float li = __shfl_sync(0xffffffffu, l, i);
            col[i] = (i > k) ? __fmaf_rn(-li, l, col[i]) : col[i];
            Lc[i] = (j == k) ? ((i == k) ? lkk : li) : Lc[i];
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) col[i] = (i == k) ? ((j == k) ? lkk : l) : col[i];
    }
    const int gst = __shfl_sync(0xffffffffu, st, 0);
    if (gst != ST_OK) {
        if (lane == 0) {
            a.status[gp] = gst;
            a.rnorm[gp] = __longlong_as_double(0x7ff8000000000000ll);
        }
        for (int c = lane; c < G + G * G; c += 32) {
            if (c < G) a.Pbar[(int64_t)gp * G + c] = __longlong_as_double(0x7ff8000000000000ll);
            else a.dPdF[(int64_t)gp * G * G + c - G] = __longlong_as_double(0x7ff8000000000000ll);
        }
        return gst;
    }
    // ---- backward, column-oriented: s = L^-T y and X = L^-T Z^T (Z = coupling
    // rows of L).  Lane i updates its right-hand side with L[k][i] = Lc[k] of
    // lane i (its own column of L) and the broadcast solution entry k.
    df sj = y;
    float xj[G];
#pragma unroll
    for (int c = 0; c < G; ++c) xj[c] = (j < n) ? sel(Lc, n + c) : 0.0f;  // Z[c][j]
    for (int k = n - 1; k >= 0; --k) {
        const float lkk = __shfl_sync(0xffffffffu, sel(Lc, k), k);
        const float inv = 1.0f / lkk;
        const df sk = df_div_f(shfl_df(sj, k), lkk, inv);
        const float lki = (j < k) ? sel(Lc, k) : 0.0f;  // L[k][j]
        if (j < k) sj = df_sub(sj, df_mul_f(sk, lki));
        if (j == k) sj = sk;
#pragma unroll
        for (int c = 0; c < G; ++c) {
            const float xk = __shfl_sync(0xffffffffu, xj[c], k) * inv;
            if (j < k) xj[c] = __fmaf_rn(-lki, xk, xj[c]);
            if (j == k) xj[c] = xk;
        }
    }
    // ---- outputs
    if (j < a.nmax) {
        const int64_t base = (int64_t)gp * a.nmax + j;
        const bool in = j < n;
        a.q[base] = in ? qd[j] : 0.0;
        a.s[base] = in ? df_to(sj) : 0.0;
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            int i1, j1;
            voigt_pair(D, v, i1, j1);
            const float sv = (i1 == j1) ? xj[i1 * D + j1] : xj[i1 * D + j1] + xj[j1 * D + i1];
            a.S[base * NS + v] = in ? (double)sv : 0.0;
        }
    }
    for (int jj = 32 + lane; jj < a.nmax; jj += 32) {        // state padding beyond one warp
        const int64_t base = (int64_t)gp * a.nmax + jj;
        a.q[base] = 0.0;
        a.s[base] = 0.0;
        for (int v = 0; v < NS; ++v) a.S[base * NS + v] = 0.0;
    }
    float rmax = fabsf(rj);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
    // Pbar_alg (double-float, lanes n..n+G-1) and C_U (trailing columns)
    df Pd[G];
    float Pa[G], CU[G * G];
#pragma unroll
    for (int c = 0; c < G; ++c) {
        Pd[c] = shfl_df(y, n + c);
        Pa[c] = Pd[c].hi * V0inv;
#pragma unroll
        for (int e = 0; e < G; ++e) CU[c * G + e] = __shfl_sync(0xffffffffu, sel(col, n + c), n + e) * V0inv;
    }
    float R[G], U[G];
#pragma unroll
    for (int c = 0; c < G; ++c) {
        R[c] = (float)Rm[c];
        U[c] = (float)Um[c];
    }
    if (lane == 0) {
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
    if (lane < G) {
        const int i0 = lane / D, J0 = lane % D;
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
                a.dPdF[((int64_t)gp * G + i * D + J) * G + lane] = (double)v;
            }
    }
    return ST_OK;
}

// ---------------------------------------------------------------------------
// shared-memory plan of the evaluation kernel (MIX: float32 contraction with
// double-float kinematics/law/residual; otherwise everything float64)
template <int D, int NA, int TA, int TB, int NP, int CI, typename KT, bool SYM = false>
struct Plan {
    static constexpr bool MIX = std::is_same<KT, float>::value;
    static constexpr int G = D * D;
    static constexpr int NS = Dims<D>::NS;
    static constexpr int NQ = NA - G;                 // largest n~ served
    static constexpr int QP = NQ | 1;                 // odd row pitch (banks)
    static constexpr int BP = NQ | 1;
    // register tiles per point: all (NA/TA)^2 blocks, or with SYM only the
    // lower blocks (the augmented system is symmetric)
    static constexpr int TPP = SYM ? (NA / TA) * (NA / TA + 1) / 2 : (NA / TA) * (NA / TB);
    static constexpr int NTILE = NP * TPP;            // tile threads
    static constexpr int NT = ((NTILE > NP * CI ? NTILE : NP * CI) + 31) / 32 * 32;  // threads per CTA
    static constexpr int KC = CI * G;                 // contraction length per chunk
    static constexpr int RPT = (NP * NQ + NT - 1) / NT;
    static_assert(NA % TA == 0 && NA % TB == 0, "tile must divide NA");
    static_assert(!SYM || TA == TB, "symmetric blocks must be square");
    static_assert(NT % 32 == 0 && NT <= 1024, "bad thread count");
    // 8-byte words (a double, or a double-float pair hi|lo stored as two
    // float arrays of the same length inside the region)
    static constexpr int o_q = 0;
    static constexpr int o_U = o_q + NP * QP;
    static constexpr int o_Udf = o_U + NP * G;
    static constexpr int o_R = o_Udf + NP * G;
    static constexpr int o_dU = o_R + NP * G;
    static constexpr int o_r = o_dU + NP * NS;
    static constexpr int o_PU = o_r + NP * NQ;
    static constexpr int o_B = o_PU + NP * G;
    static constexpr int o_WP = o_B + CI * G * BP;
    static constexpr int o_w = o_WP + NP * CI * G;
    static constexpr int o_y = o_w + CI;
    static constexpr int o_X = o_y + NP * NA;
    static constexpr int o_q64 = o_X + NP * G * NQ;   // float64 q (MIX keeps split copies in o_q)
    static constexpr int o_B2 = o_q64 + NP * QP;       // MIX: second staging buffer (Bh | Bl)
    static constexpr int o_w2 = o_B2 + (MIX ? CI * G * BP : 0);
    static constexpr int n_dbl = o_w2 + (MIX ? CI : 0);
    // ints
    static constexpr int o_ph = 0;                    // [2][CI] (MIX double-buffers)
    static constexpr int o_flag = o_ph + 2 * CI;
    static constexpr int o_pidx = o_flag + NP;
    static constexpr int n_int = ((o_pidx + NP + 3) / 4) * 4;
    // KT arrays
    static constexpr int o_Bx = 0;                    // [MIX ? 2 : 1][KC][NA]
    static constexpr int o_YM = o_Bx + (MIX ? 2 : 1) * KC * NA;
    static constexpr int NAP = NA + 1;                 // padded Y row (bank conflicts)
    static constexpr int n_YM = (NP * KC * NAP > NP * NA * NA) ? NP * KC * NAP : NP * NA * NA;
    static constexpr int n_kt = o_YM + n_YM;
    static constexpr size_t bytes = sizeof(double) * n_dbl + sizeof(int) * n_int + sizeof(KT) * n_kt;
};

// ---------------------------------------------------------------------------
template <int D, int NA, int TA, int TB, int NP, int CI, typename KT, bool ADJ, bool SYM = false>
__global__ void __launch_bounds__(Plan<D, NA, TA, TB, NP, CI, KT, SYM>::NT)
    eval_kernel(EvalArgs a) {
    using PL = Plan<D, NA, TA, TB, NP, CI, KT, SYM>;
    constexpr bool MIX = PL::MIX;
    constexpr int G = PL::G, NS = PL::NS, NQ = PL::NQ, QP = PL::QP, BP = PL::BP;
    constexpr int TPP = PL::TPP, NT = PL::NT, KC = PL::KC, RPT = PL::RPT;
    constexpr int NTB = NA / TB;
    constexpr int NAP = PL::NAP;
    // one task over several lanes in the pointwise phase of the mixed
    // configurations whose (point, ECM point) tasks fill at most half the CTA
    // (the wide ones: few points per CTA)
    constexpr bool SPLIT = MIX && !ADJ && 2 * NP * CI <= NT;
    using XT = KT;  // precision of K^-1 K_qF (feeds S and the adjoint's z)
    extern __shared__ __align__(16) unsigned char smem[];
    double *sd = reinterpret_cast<double *>(smem);
    int *si = reinterpret_cast<int *>(sd + PL::n_dbl);
    KT *sk = reinterpret_cast<KT *>(si + PL::n_int);
    double *s_q = sd + PL::o_q, *s_U = sd + PL::o_U, *s_R = sd + PL::o_R, *s_dU = sd + PL::o_dU;
    double *s_r = sd + PL::o_r, *s_PU = sd + PL::o_PU, *s_B = sd + PL::o_B, *s_WP = sd + PL::o_WP;
    double *s_w = sd + PL::o_w, *s_y = sd + PL::o_y;
    double *s_qd = MIX ? sd + PL::o_q64 : s_q;  // float64 amplitudes
    XT *s_X = reinterpret_cast<XT *>(sd + PL::o_X);
    // double-float views (MIX): hi array followed by lo array
    float *s_qh = reinterpret_cast<float *>(s_q), *s_ql = s_qh + NP * QP;
    float *s_Uh = reinterpret_cast<float *>(sd + PL::o_Udf), *s_Ul = s_Uh + NP * G;
    float *s_Bh = reinterpret_cast<float *>(s_B), *s_Bl = s_Bh + CI * G * BP;
    float *s_WPh = reinterpret_cast<float *>(s_WP), *s_WPl = s_WPh + NP * CI * G;
    float *s_wh = reinterpret_cast<float *>(s_w), *s_wl = s_wh + CI;
    int *s_ph = si + PL::o_ph, *s_flag = si + PL::o_flag, *s_pidx = si + PL::o_pidx;
    KT *s_Bx = sk + PL::o_Bx, *s_Y = sk + PL::o_YM, *s_M = sk + PL::o_YM;

    const int tid = threadIdx.x;
    const int n = a.t.n, m = a.t.m;
    const int na = n + G;
    const int64_t count = a.count ? (int64_t)(*a.count) : a.n_points;
    const int32_t *perm = a.perm ? a.perm + (a.offset ? *a.offset : 0) : nullptr;
    const int64_t n_tiles = (count + NP - 1) / NP;

    // register tile of the contraction (SYM: lower block (rb, cb), rb >= cb)
    const bool tiler = tid < PL::NTILE;
    const int tp = tiler ? tid / TPP : 0;
    const int tt = tid % TPP;
    int a0, b0;
    if (SYM) {
        int rb = 0;
        while ((rb + 1) * (rb + 2) / 2 <= tt) ++rb;
        a0 = rb * TA;
        b0 = (tt - rb * (rb + 1) / 2) * TB;
    } else {
        a0 = (tt / NTB) * TA;
        b0 = (tt % NTB) * TB;
    }
    double th[4] = {0.0, 0.0, 0.0, 0.0};  // adjoint: (mu, kappa) of phase 0, phase 1
    // material constants in double-float
    df dmu0{0.0f, 0.0f}, dmu1{0.0f, 0.0f}, dlam0{0.0f, 0.0f}, dlam1{0.0f, 0.0f};
    const KT kmu0 = (KT)a.t.mu[0], kmu1 = (KT)a.t.mu[1];
    const KT klam0 = (KT)(a.t.kappa[0] - (2.0 / 3.0) * a.t.mu[0]);
    const KT klam1 = (KT)(a.t.kappa[1] - (2.0 / 3.0) * a.t.mu[1]);
    if (MIX) {
        dmu0 = df_from(a.t.mu[0]);
        dmu1 = df_from(a.t.mu[1]);
        dlam0 = df_from(a.t.kappa[0] - (2.0 / 3.0) * a.t.mu[0]);
        dlam1 = df_from(a.t.kappa[1] - (2.0 / 3.0) * a.t.mu[1]);
    }

    if (MIX) {
        // staging buffers: zero once (entries past m keep finite values), then
        // the constant identity block of [B_i | I] in both Bx buffers
        float *b0 = reinterpret_cast<float *>(s_B), *b1 = reinterpret_cast<float *>(sd + PL::o_B2);
        for (int x = tid; x < 2 * CI * G * BP; x += NT) {
            b0[x] = 0.0f;
            b1[x] = 0.0f;
        }
        for (int x = tid; x < 2 * KC * NA; x += NT) {
            const int k = (x / NA) % KC, col = x % NA, c = k % G;
            s_Bx[x] = (col >= n && col - n == c) ? (KT)1 : (KT)0;
        }
        __syncthreads();
    }
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---- a1: polar split, micro update --------------------------------
        if (tid < NP) {
            const int p = tid;
            int64_t li = tile * NP + p;
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
                if (MIX) {
                    const df u = df_from(U[c]);
                    s_Uh[p * G + c] = u.hi;
                    s_Ul[p * G + c] = u.lo;
                }
            }
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                int i, j;
                voigt_pair(D, v, i, j);
                s_dU[p * NS + v] = (!ADJ && flag == ST_OK) ? U[i * D + j] - a.Uprev[(int64_t)gp * NS + v] : 0.0;
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
                qv = a.q[base];
                if (!ADJ) {
                    qv -= a.s[base];
#pragma unroll
                    for (int v = 0; v < NS; ++v) qv -= a.S[base * NS + v] * s_dU[p * NS + v];
                }
            }
            s_qd[p * QP + j] = qv;
            if (MIX) {
                const df v = df_from(qv);
                s_qh[p * QP + j] = v.hi;
                s_ql[p * QP + j] = v.lo;
            }
        }

        KT acc[TA][TB];
        KT kh[TA][TB], kc[TA][TB];  // MIX: Kahan-compensated sum of chunk partials
#pragma unroll
        for (int x = 0; x < TA; ++x)
#pragma unroll
            for (int y = 0; y < TB; ++y) {
                acc[x][y] = (KT)0;
                kh[x][y] = (KT)0;
                kc[x][y] = (KT)0;
            }
        double racc[RPT];
        dacc rdacc[2 * RPT];  // MIX: two independent chains per output (even / odd il)
#pragma unroll
        for (int u = 0; u < RPT; ++u) racc[u] = 0.0;
#pragma unroll
        for (int u = 0; u < 2 * RPT; ++u) rdacc[u] = dacc{0.0f, 0.0f};
        double pu = 0.0;
        df pudf = df{0.0f, 0.0f};
        __syncthreads();

        // ---- ECM loop: a2-a5 ---------------------------------------------
        // MIX: the gradient table of chunk kch+1 is copied asynchronously
        // into the other buffer while chunk kch is processed.
        auto issue_stage = [&](int buf, int i0s) {
            float *bh = reinterpret_cast<float *>(buf ? sd + PL::o_B2 : sd + PL::o_B);
            float *bl = bh + CI * G * BP;
            KT *bx = sk + PL::o_Bx + buf * KC * NA;
            float *wh = reinterpret_cast<float *>(buf ? sd + PL::o_w2 : sd + PL::o_w);
            float *wl = wh + CI;
            const int cnt = min(CI, m - i0s) * G * n;
            for (int x = tid; x < cnt; x += NT) {
                const int r = x / n, j = x - r * n;  // r = il * G + c
                const int64_t gi = (int64_t)i0s * G * n + x;
                cp_async4(bh + r * BP + j, a.t.Bh + gi);
                cp_async4(bl + r * BP + j, a.t.Bl + gi);
                cp_async4(bx + r * NA + j, a.t.Bh + gi);
            }
            if (tid < min(CI, m - i0s)) {
                cp_async4(wh + tid, a.t.wh + i0s + tid);
                cp_async4(wl + tid, a.t.wl + i0s + tid);
                cp_async4(s_ph + buf * CI + tid, a.t.phase + i0s + tid);
            }
            cp_async_commit();
        };
        if (MIX) issue_stage(0, 0);
        for (int i0 = 0, kch = 0; i0 < m; i0 += CI, ++kch) {
            const int buf = MIX ? (kch & 1) : 0;
            if (MIX) {
                if (i0 + CI < m) {
                    issue_stage(buf ^ 1, i0 + CI);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                s_Bh = buf ? reinterpret_cast<float *>(sd + PL::o_B2) : reinterpret_cast<float *>(s_B);
                s_Bl = s_Bh + CI * G * BP;
                s_wh = buf ? reinterpret_cast<float *>(sd + PL::o_w2) : reinterpret_cast<float *>(s_w);
                s_wl = s_wh + CI;
                s_Bx = sk + PL::o_Bx + buf * KC * NA;
            } else {
                // stage the chunk of the gradient table
                for (int x = tid; x < CI * G * NQ; x += NT) {
                    const int il = x / (G * NQ), rem = x % (G * NQ), c = rem / NQ, j = rem % NQ;
                    const bool in = i0 + il < m && j < n;
                    const int64_t gi = ((int64_t)(i0 + il) * G + c) * n + j;
                    s_B[(il * G + c) * BP + j] = in ? a.t.B[gi] : 0.0;
                }
                for (int x = tid; x < KC * NA; x += NT) {
                    const int k = x / NA, col = x % NA, il = k / G, c = k % G;
                    KT v = (KT)0;
                    if (i0 + il < m) {
                        const int64_t gi = ((int64_t)(i0 + il) * G + c) * n + col;
                        if (col < n) v = (KT)a.t.B[gi];
                        else if (col - n == c) v = (KT)1;
                    }
                    s_Bx[x] = v;
                }
                if (tid < CI) {
                    const bool ok = i0 + tid < m;
                    s_w[tid] = ok ? a.t.w[i0 + tid] : 0.0;
                    s_ph[tid] = ok ? a.t.phase[i0 + tid] : 0;
                }
            }
            __syncthreads();

            // pointwise: F_i, law, w P_i, Y_i = w A_i [B_i | I].
            // Wide mixed configurations (few points per CTA) spread a
            // (point, ECM point) task over LPT lanes: lane c forms component
            // F_c (double-float), the group exchanges F by shuffles, evaluates
            // the law redundantly, and lane c writes w P_c, tangent row c and
            // Y row c -- so the task count NP x CI need not fill the CTA.
            if constexpr (SPLIT) {
                constexpr int LPT = G <= 4 ? 4 : 16;
                const int c = tid % LPT;
                for (int base = 0; base < NP * CI; base += NT / LPT) {
                    const int task = base + tid / LPT;
                    const bool valid = task < NP * CI;
                    const int p = valid ? task % NP : 0, il = valid ? task / NP : 0;
                    bool live = valid && (s_flag[p] == ST_OK) && (i0 + il < m);
                    const int ph = s_ph[buf * CI + il];
                    df Fc{0.0f, 0.0f};
                    if (live && c < G) {
                        const float *Bh = s_Bh + (il * G + c) * BP, *Bl = s_Bl + (il * G + c) * BP;
                        const float *qh = s_qh + p * QP, *ql = s_ql + p * QP;
                        // four partial sums over j mod 4 (independent chains)
                        dacc s4[4] = {{s_Uh[p * G + c], s_Ul[p * G + c]}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
                        int j = 0;
                        for (; j + 4 <= n; j += 4) {
#pragma unroll
                            for (int t = 0; t < 4; ++t) dacc_fma(s4[t], Bh[j + t], Bl[j + t], qh[j + t], ql[j + t]);
                        }
                        for (; j < n; ++j) dacc_fma(s4[0], Bh[j], Bl[j], qh[j], ql[j]);
                        Fc = df_add(df_add(dacc_get(s4[0]), dacc_get(s4[1])), df_add(dacc_get(s4[2]), dacc_get(s4[3])));
                    }
                    df Pc;
                    float fif[G], lnf = 0.0f;
                    const bool lok = nh_stress_df_split<D, LPT>(Fc, c, ph ? dmu1 : dmu0, ph ? dlam1 : dlam0, Pc, fif, lnf);
                    if (live && !lok) {
                        if (c == 0) atomicCAS(&s_flag[p], ST_OK, ST_DETF);
                        live = false;  // the same J in every lane of the group: the same decision
                    }
                    if (valid && c < G) {
                        KT *yr = s_Y + ((il * G + c) * NP + p) * NAP;  // row k = il*G + c
                        if (live) {
                            KT fi[G], Ar[G];
#pragma unroll
                            for (int c2 = 0; c2 < G; ++c2) fi[c2] = (KT)fif[c2];
                            const df wp = df_mul(df{s_wh[il], s_wl[il]}, Pc);
                            s_WPh[(il * G + c) * NP + p] = wp.hi;
                            s_WPl[(il * G + c) * NP + p] = wp.lo;
                            const KT muk = ph ? kmu1 : kmu0, lam = ph ? klam1 : klam0;
                            const KT c3 = muk - lam * (KT)lnf;
                            nh_tangent_row_rt<D, KT>(fi, lam, c3, muk, c, Ar);  // row c of the tangent
                            const KT *Bx = s_Bx + il * G * NA;
                            const KT wk = (KT)s_wh[il];
                            for (int b = 0; b < n; ++b) {
                                KT v = (KT)0;
#pragma unroll
                                for (int c2 = 0; c2 < G; ++c2) v = kfma(Ar[c2], Bx[c2 * NA + b], v);
                                yr[b] = wk * v;
                            }
#pragma unroll
                            for (int c2 = 0; c2 < G; ++c2) yr[n + c2] = wk * Ar[c2];
                            for (int b = na; b < NA; ++b) yr[b] = (KT)0;
                        } else {
                            s_WPh[(il * G + c) * NP + p] = 0.0f;
                            s_WPl[(il * G + c) * NP + p] = 0.0f;
                            for (int b = 0; b < NA; ++b) yr[b] = (KT)0;
                        }
                    }
                }
            } else
            for (int task = tid; task < NP * CI; task += NT) {
                const int p = task % NP, il = task / NP;
                KT *yrow = s_Y + ((il * G) * NP + p) * NAP;  // row k = il*G + c at yrow + c*NP*NAP
                bool live = (s_flag[p] == ST_OK) && (i0 + il < m);
                const int ph = s_ph[buf * CI + il];
                KT fi[G];
                KT lnJk = (KT)0;
                if (live) {
                    if (MIX) {
                        df F[G], P[G];
                        const float *Bh = s_Bh + il * G * BP, *Bl = s_Bl + il * G * BP;
                        const float *qh = s_qh + p * QP, *ql = s_ql + p * QP;
                        dacc sacc[G];
#pragma unroll
                        for (int c = 0; c < G; ++c) sacc[c] = dacc{s_Uh[p * G + c], s_Ul[p * G + c]};
#pragma unroll 4
                        for (int j = 0; j < n; ++j) {
                            const float qhj = qh[j], qlj = ql[j];
#pragma unroll
                            for (int c = 0; c < G; ++c) dacc_fma(sacc[c], Bh[c * BP + j], Bl[c * BP + j], qhj, qlj);
                        }
#pragma unroll
                        for (int c = 0; c < G; ++c) F[c] = dacc_get(sacc[c]);
                        float lnf;
                        float fif[G];
                        if (!nh_stress_df<D>(F, ph ? dmu1 : dmu0, ph ? dlam1 : dlam0, P, fif, lnf)) {
                            atomicCAS(&s_flag[p], ST_OK, ST_DETF);
                            live = false;
                        } else {
                            const df w2{s_wh[il], s_wl[il]};
#pragma unroll
                            for (int c = 0; c < G; ++c) {
                                const df wp = df_mul(w2, P[c]);
                                s_WPh[(il * G + c) * NP + p] = wp.hi;
                                s_WPl[(il * G + c) * NP + p] = wp.lo;
                                fi[c] = (KT)fif[c];
                            }
                            lnJk = (KT)lnf;
                        }
                    } else {
                        double F[G], P[G], Fi[G], lnJ = 0.0;
                        const double *Bi = s_B + il * G * BP;
                        const double *qp = s_q + p * QP;
#pragma unroll
                        for (int c = 0; c < G; ++c) F[c] = s_U[p * G + c];
                        for (int j = 0; j < n; ++j) {
                            const double qj = qp[j];
#pragma unroll
                            for (int c = 0; c < G; ++c) F[c] = fma(Bi[c * BP + j], qj, F[c]);
                        }
                        if (!nh_stress<D>(F, a.t.mu[ph], a.t.kappa[ph], P, Fi, lnJ)) {
                            atomicCAS(&s_flag[p], ST_OK, ST_DETF);
                            live = false;
                        } else {
                            const double wi = s_w[il];
#pragma unroll
                            for (int c = 0; c < G; ++c) {
                                s_WP[(il * G + c) * NP + p] = wi * P[c];
                                fi[c] = (KT)Fi[c];
                            }
                            lnJk = (KT)lnJ;
                        }
                    }
                }
                if (live) {
                    const KT muk = ph ? kmu1 : kmu0, lam = ph ? klam1 : klam0;
                    const KT c3 = muk - lam * lnJk;
                    const KT *Bx = s_Bx + il * G * NA;
                    const KT wk = MIX ? (KT)s_wh[il] : (KT)s_w[il];
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        KT Ar[G];
                        nh_tangent_row<D, KT>(fi, lam, c3, muk, c, Ar);
                        KT *yr = yrow + c * NP * NAP;
                        for (int b = 0; b < n; ++b) {
                            KT v = (KT)0;
#pragma unroll
                            for (int c2 = 0; c2 < G; ++c2) v = kfma(Ar[c2], Bx[c2 * NA + b], v);
                            yr[b] = wk * v;
                        }
#pragma unroll
                        for (int c2 = 0; c2 < G; ++c2) yr[n + c2] = wk * Ar[c2];
                        for (int b = na; b < NA; ++b) yr[b] = (KT)0;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        if (MIX) {
                            s_WPh[(il * G + c) * NP + p] = 0.0f;
                            s_WPl[(il * G + c) * NP + p] = 0.0f;
                        } else {
                            s_WP[(il * G + c) * NP + p] = 0.0;
                        }
                        KT *yr = yrow + c * NP * NAP;
                        for (int b = 0; b < NA; ++b) yr[b] = (KT)0;
                    }
                }
            }
            __syncthreads();

            // contraction of the augmented system (register tiles)
            if (tiler) {
                const KT *Yp = s_Y + tp * NAP + b0;
#pragma unroll 4
                for (int k = 0; k < KC; ++k) {
                    KT av[TA], bv[TB];
#pragma unroll
                    for (int x = 0; x < TA; ++x) av[x] = s_Bx[k * NA + a0 + x];
#pragma unroll
                    for (int y = 0; y < TB; ++y) bv[y] = Yp[k * NP * NAP + y];
#pragma unroll
                    for (int x = 0; x < TA; ++x)
#pragma unroll
                        for (int y = 0; y < TB; ++y) acc[x][y] = kfma(av[x], bv[y], acc[x][y]);
                }
                if (MIX) {
                    // fold the chunk partial into the compensated sum
#pragma unroll
                    for (int x = 0; x < TA; ++x)
#pragma unroll
                        for (int y = 0; y < TB; ++y) {
                            const float yv = __fsub_rn(acc[x][y], kc[x][y]);
                            const float t = __fadd_rn(kh[x][y], yv);
                            kc[x][y] = __fsub_rn(__fsub_rn(t, kh[x][y]), yv);
                            kh[x][y] = t;
                            acc[x][y] = 0.0f;
                        }
                }
            }
            // float64-accurate reduced residual and homogenized stress
            if (MIX) {
                // all of this thread's rows at once (2 RPT independent chains);
                // a row past the CTA's points reads row 0 and is never stored,
                // rows j >= n are stored as zero
                int bo[RPT], wo[RPT];
#pragma unroll
                for (int u = 0; u < RPT; ++u) {
                    const int o = tid + u * NT;
                    const bool in = o < NP * NQ;
                    wo[u] = in ? o / NQ : 0;
                    bo[u] = in ? o % NQ : 0;
                }
                for (int il = 0; il < CI; il += 2)
#pragma unroll
                    for (int c = 0; c < G; ++c)
#pragma unroll
                        for (int u = 0; u < RPT; ++u) {
                            const int b0 = (il * G + c) * BP + bo[u], w0 = (il * G + c) * NP + wo[u];
                            const int b1 = b0 + G * BP, w1 = w0 + G * NP;
                            dacc_fma(rdacc[2 * u], s_Bh[b0], s_Bl[b0], s_WPh[w0], s_WPl[w0]);
                            dacc_fma(rdacc[2 * u + 1], s_Bh[b1], s_Bl[b1], s_WPh[w1], s_WPl[w1]);
                        }
            } else {
#pragma unroll
                for (int u = 0; u < RPT; ++u) {
                    const int o = tid + u * NT;
                    if (o < NP * NQ) {
                        const int p = o / NQ, j = o % NQ;
                        if (j < n) {
                            double v = racc[u];
                            for (int il = 0; il < CI; ++il)
#pragma unroll
                                for (int c = 0; c < G; ++c)
                                    v = fma(s_B[(il * G + c) * BP + j], s_WP[(il * G + c) * NP + p], v);
                            racc[u] = v;
                        }
                    }
                }
            }
            if (tid < NP * G) {
                const int p = tid / G, c = tid % G;
                for (int il = 0; il < CI; ++il) {
                    if (MIX) pudf = df_add(pudf, df{s_WPh[(il * G + c) * NP + p], s_WPl[(il * G + c) * NP + p]});
                    else pu += s_WP[(il * G + c) * NP + p];
                }
            }
            __syncthreads();
        }

        // ---- spill accumulators for the condensation ----------------------
        // (MIX keeps r and V0 Pbar_U as double-float pairs: hi in the first,
        // lo in the second half of the float view of s_r / s_PU)
        float *s_rh = reinterpret_cast<float *>(s_r), *s_rl = s_rh + NP * NQ;
        float *s_puh = reinterpret_cast<float *>(s_PU), *s_pul = s_puh + NP * G;
        if (tiler) {
#pragma unroll
            for (int x = 0; x < TA; ++x)
#pragma unroll
                for (int y = 0; y < TB; ++y)
                    s_M[(tp * NA + a0 + x) * NA + b0 + y] = MIX ? (KT)(kh[x][y] - kc[x][y]) : acc[x][y];
        }
        if (MIX) {
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int o = tid + u * NT;
                if (o < NP * NQ) {
                    const df v = (o % NQ) < n ? df_add(dacc_get(rdacc[2 * u]), dacc_get(rdacc[2 * u + 1])) : df{0.0f, 0.0f};
                    s_rh[o] = v.hi;
                    s_rl[o] = v.lo;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int o = tid + u * NT;
                if (o < NP * NQ) s_r[o] = racc[u];
            }
        }
        if (tid < NP * G) {
            if (MIX) {
                s_puh[tid] = pudf.hi;
                s_pul[tid] = pudf.lo;
            } else {
                s_PU[tid] = pu;
            }
        }
        __syncthreads();
        // ---- a6: condensation, one warp per point --------------------------
        const int warp = tid >> 5, lane = tid & 31;
        constexpr bool REGS = MIX && NA <= 32 && !ADJ;
        if (REGS) {
            for (int p = warp; p < NP; p += NT / 32) {
                const int gp = s_pidx[p];
                if (gp < 0) continue;
                condense_out_regs_mix<D, (NA <= 32 ? NA : 32), NQ>(
                    a, reinterpret_cast<const float *>(s_M + p * NA * NA), s_rh + p * NQ, s_rl + p * NQ,
                    s_puh + p * G, s_pul + p * G, gp, s_flag[p], n, s_qd + p * QP, s_R + p * G, s_U + p * G,
                    (float)(1.0 / a.V0), lane);
            }
        }
        for (int p = warp; p < NP && !REGS; p += NT / 32) {
            if (s_flag[p] != ST_OK) continue;
            int st;
            if (MIX) {
                float *yh = reinterpret_cast<float *>(s_y + p * NA);
                st = condense_warp_mix<D, NA, NQ>(reinterpret_cast<float *>(s_M + p * NA * NA), yh, yh + NA,
                                                  reinterpret_cast<float *>(s_X + p * G * NQ), s_rh + p * NQ,
                                                  s_rl + p * NQ, s_puh + p * G, s_pul + p * G, n, lane);
            } else {
                st = condense_warp<D, NA, NQ, KT, XT>(s_M + p * NA * NA, s_y + p * NA, s_X + p * G * NQ,
                                                    s_r + p * NQ, s_PU + p * G, n, lane);
            }
            if (lane == 0 && st != ST_OK) s_flag[p] = st;
        }
        __syncthreads();

        // ---- a7: outputs ---------------------------------------------------
        for (int p = warp; p < NP && !ADJ && !REGS; p += NT / 32) {
            const int gp = s_pidx[p];
            if (gp < 0) continue;
            if (MIX) {
                const float *yh = reinterpret_cast<const float *>(s_y + p * NA);
                write_outputs_warp_mix<D, NA, NQ>(a, gp, s_flag[p], n, yh, yh + NA,
                                                  reinterpret_cast<const float *>(s_X + p * G * NQ),
                                                  reinterpret_cast<const float *>(s_M + p * NA * NA),
                                                  s_qd + p * QP, s_rh + p * NQ, s_R + p * G, s_U + p * G,
                                                  (float)(1.0 / a.V0), lane);
            } else {
                write_outputs_warp<D, NA, NQ, KT, XT>(a, gp, s_flag[p], n, s_y + p * NA, s_X + p * G * NQ,
                                                    s_M + p * NA * NA, s_qd + p * QP, s_r + p * NQ, s_R + p * G,
                                                    s_U + p * G, lane);
            }
        }
        __syncthreads();

        if (ADJ) {
            // cotangent on Fbar through the condensed tangent, and z = K^-1 K_qF R^T gP
            for (int p = warp; p < NP; p += NT / 32) {
                const int gp = s_pidx[p];
                if (gp < 0) continue;
                const int flag = s_flag[p];
                double *y = s_y + p * NA;
                const XT *X = s_X + p * G * NQ;
                const KT *M = s_M + p * NA * NA;
                if (flag != ST_OK) {
                    if (lane == 0) {
                        a.status[gp] = flag;
                        for (int c = 0; c < G; ++c) a.gF[(int64_t)gp * G + c] = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
                        for (int c = 0; c < G; ++c) s_PU[p * G + c] = 0.0;
                    }
                    for (int j = lane; j < NQ; j += 32) y[j] = 0.0;
                    continue;
                }
                double gPU[G];
                {
                    double gPv[G], R[G];
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        gPv[c] = a.gP[(int64_t)gp * G + c];
                        R[c] = s_R[p * G + c];
                    }
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int J = 0; J < D; ++J) {
                            double v = 0.0;
#pragma unroll
                            for (int k = 0; k < D; ++k) v += R[k * D + i] * gPv[k * D + J];
                            gPU[i * D + J] = v;
                        }
                    if (lane == 0) {
                        a.status[gp] = ST_OK;
                        const double iV = 1.0 / a.V0;
                        double Pa[G], U[G], CU[G * G];
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            Pa[c] = y[n + c] * iV;
                            U[c] = s_U[p * G + c];
                        }
#pragma unroll
                        for (int c = 0; c < G; ++c)
#pragma unroll
                            for (int e = 0; e < G; ++e) {
                                const int hi = c > e ? c : e, lo = c > e ? e : c;
                                CU[c * G + e] = (double)M[(n + hi) * NA + n + lo] * iV;
                            }
                        // gF[e] = sum_c dPdF[c][e] gP[c], column e from the polar derivative
#pragma unroll
                        for (int i0 = 0; i0 < D; ++i0)
#pragma unroll
                            for (int J0 = 0; J0 < D; ++J0) {
                                double Om[G], dU[G], T[G];
                                polar_dir<D>(R, U, i0, J0, Om, dU);
#pragma unroll
                                for (int c = 0; c < G; ++c) {
                                    double v = 0.0;
#pragma unroll
                                    for (int e = 0; e < G; ++e) v += CU[c * G + e] * dU[e];
                                    T[c] = v;
                                }
#pragma unroll
                                for (int i = 0; i < D; ++i)
#pragma unroll
                                    for (int J = 0; J < D; ++J) {
                                        double v = T[i * D + J];
#pragma unroll
                                        for (int k = 0; k < D; ++k) v += Om[i * D + k] * Pa[k * D + J];
                                        T[i * D + J] = v;
                                    }
                                // <gP, R T> = <R^T gP, T>
                                double v = 0.0;
#pragma unroll
                                for (int c = 0; c < G; ++c) v += gPU[c] * T[c];
                                a.gF[(int64_t)gp * G + i0 * D + J0] = v;
                            }
                    }
                }
                __syncwarp();
                // z_j = sum_c X[c][j] gPU[c]  (stored over y[0:n))
                for (int j = lane; j < NQ; j += 32) {
                    double v = 0.0;
                    if (j < n)
#pragma unroll
                        for (int c = 0; c < G; ++c) v += (double)X[c * NQ + j] * gPU[c];
                    y[j] = v;
                }
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < G; ++c) s_PU[p * G + c] = gPU[c];
            }
            __syncthreads();
            // second pass over the ECM points: (1/V0) w_i <gPU - B_i z, dP_i/dtheta>
            for (int i0 = 0; i0 < m; i0 += CI) {
                for (int x = tid; x < CI * G * NQ; x += NT) {
                    const int il = x / (G * NQ), rem = x % (G * NQ), c = rem / NQ, j = rem % NQ;
                    double v = 0.0;
                    if (i0 + il < m && j < n) v = a.t.B[((int64_t)(i0 + il) * G + c) * n + j];
                    s_B[(il * G + c) * BP + j] = v;
                }
                if (tid < CI) {
                    const bool ok = i0 + tid < m;
                    s_w[tid] = ok ? a.t.w[i0 + tid] : 0.0;
                    s_ph[tid] = ok ? a.t.phase[i0 + tid] : 0;
                }
                __syncthreads();
                for (int task = tid; task < NP * CI; task += NT) {
                    const int p = task % NP, il = task / NP;
                    if (s_flag[p] != ST_OK || i0 + il >= m) continue;
                    const double *Bi = s_B + il * G * BP;
                    const double *qp = s_qd + p * QP;
                    const double *zp = s_y + p * NA;
                    double F[G], Fi[G], v[G];
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        double f = s_U[p * G + c], bz = 0.0;
                        for (int j = 0; j < n; ++j) {
                            f = fma(Bi[c * BP + j], qp[j], f);
                            bz = fma(Bi[c * BP + j], zp[j], bz);
                        }
                        F[c] = f;
                        v[c] = s_PU[p * G + c] - bz;
                    }
                    const double J = inverse<D>(F, Fi);
                    const double lnJ = log(J);
                    double dmu = 0.0, dka = 0.0;
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int Jc = 0; Jc < D; ++Jc) {
                            const double fit = Fi[Jc * D + i];
                            const double vc = v[i * D + Jc];
                            dmu += vc * (F[i * D + Jc] - fit - (2.0 / 3.0) * lnJ * fit);
                            dka += vc * (lnJ * fit);
                        }
                    const double wv = s_w[il] / a.V0;
                    const int ph = s_ph[il];
                    th[2 * ph] += wv * dmu;
                    th[2 * ph + 1] += wv * dka;
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
    if (ADJ) {
        // deterministic block reduction of the moduli gradient into partials
        double *red = reinterpret_cast<double *>(smem);
        for (int k = 0; k < 4; ++k) {
            double v = th[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if ((tid & 31) == 0) red[(tid >> 5) * 4 + k] = v;
        }
        __syncthreads();
        if (tid < 4) {
            double v = 0.0;
            for (int w = 0; w < NT / 32; ++w) v += red[w * 4 + tid];
            a.partials[(int64_t)blockIdx.x * 4 + tid] = v;
        }
    }
}

}  // namespace rverom
