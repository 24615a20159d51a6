// rverom_j2.cu -- the hyper-reduced RVE evaluation with a history-dependent
// micro law at the ECM points (steps a1-a7 of rve_rom_eval_batch, float64):
// small-strain J2 plasticity with linear isotropic hardening, the matrix law
// of Example 1 (Sec. 5.1), under plane strain, one history record per ECM
// point and macro point.
//
// Law at an ECM point (radial return, backward Euler; eps = sym(F - I) with
// eps_33 = 0, records [eps_p 11, 22, 33, 12, 13, 23, alpha] of the last
// converged load step):
//   s_tr = 2 mu (dev eps - eps_p),  f = |s_tr| - sqrt(2/3) (sy0 + h alpha)
//   f <= 0:  sigma = kappa tr(eps) I + s_tr,  C = kappa I(x)I + 2 mu I_dev
//   else:    dgam = f / (2 mu + 2 h / 3),  n = s_tr / |s_tr|,
//            sigma = kappa tr(eps) I + s_tr - 2 mu dgam n,
//            eps_p += dgam n,  alpha += sqrt(2/3) dgam,
//            C = kappa I(x)I + 2 mu b I_dev - 2 mu c n(x)n,
//            b = 1 - 2 mu dgam / |s_tr|,  c = 1 / (1 + h / (3 mu)) - (1 - b)
// The in-plane stress takes the place of P and the in-plane block of C that
// of dP/dF in the reduced residual, stiffness and condensation.
//
// One warp per macro point: lanes take 32 ECM points at a time (kinematics,
// return mapping, w_i P_i and Y_i = w_i A_i [B_i | I] into shared memory),
// then the lanes own entries of the lower triangle of the augmented system
// M = sum_i [B_i | I]^T Y_i and of the residual; the condensation and the
// outputs are those of the float64 Neo-Hooke form (condense_warp,
// write_outputs_warp).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/rverom.h"
#include "rverom_internal.h"

namespace rverom {
namespace {

constexpr int J2_NH = 7;      // history words per ECM point
constexpr int J2_WARPS = 4;   // warps (points in flight) per CTA
constexpr int J2_CH = 32;     // ECM points per chunk (one per lane)

struct J2Args {
    const double *hist_in;
    double *hist_out;
    int mmax;                  // ECM-point stride of the history arrays
    double sy0[2], hk[2];      // yield stress, hardening modulus per phase
};

template <int NA>
struct J2Plan {
    static constexpr int G = 4, NQ = NA - G;
    static constexpr int NL = NA * (NA + 1) / 2;        // lower triangle of M
    static constexpr int NE = (NL + 31) / 32;            // entries per lane
    static constexpr int o_Y = 0;                        // [CH][G][NA]
    static constexpr int o_wP = o_Y + J2_CH * G * NA;    // [CH][G]
    static constexpr int o_M = o_wP + J2_CH * G;         // [NA][NA]
    static constexpr int o_y = o_M + NA * NA;            // [NA]
    static constexpr int o_X = o_y + NA;                 // [G][NQ]
    static constexpr int o_r = o_X + G * NQ;             // [NQ]
    static constexpr int o_PU = o_r + NQ;                // [G]
    static constexpr int o_q = o_PU + G;                 // [NQ]
    static constexpr int o_R = o_q + NQ;                 // [G]
    static constexpr int o_U = o_R + G;                  // [G]
    static constexpr int WORDS = o_U + G;                // doubles per warp
    static constexpr size_t bytes = (size_t)WORDS * J2_WARPS * sizeof(double);
};

// plane-strain J2 return mapping; eps2 = in-plane symmetric strain (11, 22,
// 12); returns the in-plane stress (2 x 2, row-major) and tangent (4 x 4 over
// the in-plane components), updates rec[7]
__device__ void j2_point(const double *eps2, double mu, double kappa, double sy0, double hk, const double *rec_in,
                         double *rec_out, double *P, double *A) {
    // 3D strain and its deviator (eps_33 = 0)
    const double e11 = eps2[0], e22 = eps2[1], e12 = eps2[2];
    const double tr = e11 + e22;
    double dv[6] = {e11 - tr / 3.0, e22 - tr / 3.0, -tr / 3.0, e12, 0.0, 0.0};
    double st[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) st[k] = 2.0 * mu * (dv[k] - rec_in[k]);
    // |s|^2 with the shear entries counted twice
    const double nrm = sqrt(st[0] * st[0] + st[1] * st[1] + st[2] * st[2] +
                            2.0 * (st[3] * st[3] + st[4] * st[4] + st[5] * st[5]));
    const double alpha = rec_in[6];
    const double f = nrm - sqrt(2.0 / 3.0) * (sy0 + hk * alpha);
    double b = 1.0, c = 0.0, nn[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < J2_NH; ++k) rec_out[k] = rec_in[k];
    double s[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = st[k];
    if (isfinite(sy0) && f > 0.0) {
        const double dg = f / (2.0 * mu + 2.0 * hk / 3.0);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            nn[k] = st[k] / nrm;
            s[k] = st[k] - 2.0 * mu * dg * nn[k];
            rec_out[k] = rec_in[k] + dg * nn[k];
        }
        rec_out[6] = alpha + sqrt(2.0 / 3.0) * dg;
        b = 1.0 - 2.0 * mu * dg / nrm;
        c = 1.0 / (1.0 + hk / (3.0 * mu)) - (1.0 - b);
    }
    // in-plane stress: sigma_ij = kappa tr d_ij + s_ij
    P[0] = kappa * tr + s[0];
    P[1] = s[3];
    P[2] = s[3];
    P[3] = kappa * tr + s[1];
    // tangent C_iJkL = kappa d_iJ d_kL + 2 mu b (Isym - IxI/3)_iJkL - 2 mu c n_iJ n_kL
    // over in-plane components c = i*2 + J (n in full 3 x 3 form: n_01 = n_10 = nn[3])
    const double n2[4] = {nn[0], nn[3], nn[3], nn[1]};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = p / 2, J = p % 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = q / 2, L = q % 2;
            const double dij = (i == J) ? 1.0 : 0.0, dkl = (k == L) ? 1.0 : 0.0;
            const double isym = 0.5 * (((i == k) && (J == L) ? 1.0 : 0.0) + ((i == L) && (J == k) ? 1.0 : 0.0));
            A[p * 4 + q] = kappa * dij * dkl + 2.0 * mu * b * (isym - dij * dkl / 3.0) - 2.0 * mu * c * n2[p] * n2[q];
        }
    }
}

template <int NA>
__global__ void __launch_bounds__(J2_WARPS * 32) eval_j2_kernel(EvalArgs a, J2Args j) {
    using PL = J2Plan<NA>;
    constexpr int G = PL::G, NQ = PL::NQ, NS = 3, NE = PL::NE;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *base = reinterpret_cast<double *>(smem) + (size_t)warp * PL::WORDS;
    double *Y = base + PL::o_Y, *wP = base + PL::o_wP, *M = base + PL::o_M, *y = base + PL::o_y;
    double *X = base + PL::o_X, *r = base + PL::o_r, *PU = base + PL::o_PU, *qd = base + PL::o_q;
    double *Rm = base + PL::o_R, *Um = base + PL::o_U;
    const int n = a.t.n, m = a.t.m, na = n + G;
    const int64_t count = a.count ? (int64_t)(*a.count) : a.n_points;
    const int64_t off = (a.perm && a.offset) ? (int64_t)(*a.offset) : 0;
    const int32_t *perm = a.perm ? a.perm + off : nullptr;
    const int64_t gw = (int64_t)blockIdx.x * J2_WARPS + warp, nwt = (int64_t)gridDim.x * J2_WARPS;
    for (int64_t li = gw; li < count; li += nwt) {
        const int gp = perm ? perm[li] : (int)li;
        // ---- a1: polar split, micro update
        int flag = ST_OK;
        if (lane == 0) {
            double F[G], R[G], U[G];
            bool fin = true;
#pragma unroll
            for (int c = 0; c < G; ++c) {
                F[c] = a.Fbar[(int64_t)gp * G + c];
                fin = fin && isfinite(F[c]);
            }
            if (!fin) flag = ST_NONFINITE;
            else if (!(det<2>(F) > 0.0) || !polar<2>(F, R, U)) flag = ST_DETF;
#pragma unroll
            for (int c = 0; c < G; ++c) {
                Rm[c] = flag == ST_OK ? R[c] : 0.0;
                Um[c] = flag == ST_OK ? U[c] : 0.0;
            }
        }
        flag = __shfl_sync(0xffffffffu, flag, 0);
        __syncwarp();
        if (flag == ST_OK) {
            double dU[NS];
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                int i1, j1;
                voigt_pair(2, v, i1, j1);
                dU[v] = Um[i1 * 2 + j1] - a.Uprev[(int64_t)gp * NS + v];
            }
            for (int jj = lane; jj < n; jj += 32) {
                const int64_t b = (int64_t)gp * a.nmax + jj;
                double v = a.q[b] - a.s[b];
#pragma unroll
                for (int k = 0; k < NS; ++k) v -= a.S[b * NS + k] * dU[k];
                qd[jj] = v;
            }
        }
        __syncwarp();
        // ---- a2-a5 by chunks of 32 ECM points
        double macc[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) macc[e] = 0.0;
        double racc[(NQ + 31) / 32];
#pragma unroll
        for (int e = 0; e < (NQ + 31) / 32; ++e) racc[e] = 0.0;
        double pacc = 0.0;
        bool bad = false;
        for (int c0 = 0; c0 < m && flag == ST_OK; c0 += J2_CH) {
            const int i = c0 + lane;
            if (i < m) {
                const double *Bi = a.t.B + (int64_t)i * G * n;
                double F[G];
#pragma unroll
                for (int c = 0; c < G; ++c) {
                    double v = Um[c];
                    for (int k = 0; k < n; ++k) v += Bi[c * n + k] * qd[k];
                    F[c] = v;
                }
                bad = bad || !(det<2>(F) > 0.0);
                const int ph = a.t.phase[i];
                const double eps2[3] = {F[0] - 1.0, F[3] - 1.0, 0.5 * (F[1] + F[2])};
                double P[G], A[G * G];
                const int64_t hb = ((int64_t)gp * j.mmax + i) * J2_NH;
                double rin[J2_NH], rout[J2_NH];
#pragma unroll
                for (int k = 0; k < J2_NH; ++k) rin[k] = j.hist_in[hb + k];
                j2_point(eps2, a.t.mu[ph], a.t.kappa[ph], j.sy0[ph], j.hk[ph], rin, rout, P, A);
#pragma unroll
                for (int k = 0; k < J2_NH; ++k) j.hist_out[hb + k] = rout[k];
                const double w = a.t.w[i];
#pragma unroll
                for (int c = 0; c < G; ++c) wP[lane * G + c] = w * P[c];
                // Y_i[c][c'] = w sum_e A[c][e] Bext_i[e][c'],  Bext_i = [B_i | I]
                for (int cp = 0; cp < NA; ++cp) {
#pragma unroll
                    for (int c = 0; c < G; ++c) {
                        double v = 0.0;
                        if (cp < n) {
#pragma unroll
                            for (int e = 0; e < G; ++e) v += A[c * G + e] * Bi[e * n + cp];
                        } else if (cp < na) {
                            v = A[c * G + (cp - n)];
                        }
                        Y[(lane * G + c) * NA + cp] = w * v;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < G; ++c) wP[lane * G + c] = 0.0;
                for (int x = 0; x < G * NA; ++x) Y[lane * G * NA + x] = 0.0;
            }
            __syncwarp();
            const int nl = (m - c0) < J2_CH ? (m - c0) : J2_CH;
            // M[jj][kk] (kk <= jj) += sum_l sum_c Bext_l[c][jj] Y_l[c][kk]
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int t = lane + 32 * e;
                if (t < PL::NL) {
                    int jj = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
                    while (jj * (jj + 1) / 2 > t) --jj;
                    while ((jj + 1) * (jj + 2) / 2 <= t) ++jj;
                    const int kk = t - jj * (jj + 1) / 2;
                    double v = 0.0;
                    for (int l = 0; l < nl; ++l) {
                        const double *Bl = a.t.B + (int64_t)(c0 + l) * G * n;
#pragma unroll
                        for (int c = 0; c < G; ++c) {
                            const double bx = jj < n ? Bl[c * n + jj] : (jj - n == c ? 1.0 : 0.0);
                            v += bx * Y[(l * G + c) * NA + kk];
                        }
                    }
                    macc[e] += v;
                }
            }
            // r[jj] += sum_l sum_c B_l[c][jj] wP_l[c];  V0 Pbar_U[c] += sum_l wP_l[c]
#pragma unroll
            for (int e = 0; e < (NQ + 31) / 32; ++e) {
                const int jj = lane + 32 * e;
                if (jj < n) {
                    double v = 0.0;
                    for (int l = 0; l < nl; ++l) {
                        const double *Bl = a.t.B + (int64_t)(c0 + l) * G * n;
#pragma unroll
                        for (int c = 0; c < G; ++c) v += Bl[c * n + jj] * wP[l * G + c];
                    }
                    racc[e] += v;
                }
            }
            if (lane < G)
                for (int l = 0; l < nl; ++l) pacc += wP[l * G + lane];
            __syncwarp();
        }
        if (flag == ST_OK && __any_sync(0xffffffffu, bad)) flag = ST_DETF;
        if (flag == ST_OK) {
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int t = lane + 32 * e;
                if (t < PL::NL) {
                    int jj = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
                    while (jj * (jj + 1) / 2 > t) --jj;
                    while ((jj + 1) * (jj + 2) / 2 <= t) ++jj;
                    const int kk = t - jj * (jj + 1) / 2;
                    M[jj * NA + kk] = macc[e];
                }
            }
#pragma unroll
            for (int e = 0; e < (NQ + 31) / 32; ++e) {
                const int jj = lane + 32 * e;
                if (jj < n) r[jj] = racc[e];
            }
            if (lane < G) PU[lane] = pacc;
            __syncwarp();
            flag = condense_warp<2, NA, NQ, double, double>(M, y, X, r, PU, n, lane);
        }
        if (flag != ST_OK) {
            // a failed point keeps its history (as it keeps its micro state)
            for (int x = lane; x < m * J2_NH; x += 32) {
                const int64_t hb = (int64_t)gp * j.mmax * J2_NH + x;
                j.hist_out[hb] = j.hist_in[hb];
            }
        }
        __syncwarp();
        write_outputs_warp<2, NA, NQ, double, double>(a, gp, flag, n, y, X, M, qd, r, Rm, Um, lane);
        __syncwarp();
    }
}

template <int NA>
cudaError_t launch_j2(const EvalArgs &a, const J2Args &j, int n_sm, int64_t max_points, cudaStream_t st) {
    using PL = J2Plan<NA>;
    auto kern = eval_j2_kernel<NA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, J2_WARPS * 32, PL::bytes);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t grid = (max_points + J2_WARPS - 1) / J2_WARPS;
    if (grid > (int64_t)n_sm * occ) grid = (int64_t)n_sm * occ;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, J2_WARPS * 32, PL::bytes, st>>>(a, j);
    return cudaGetLastError();
}

}  // namespace
}  // namespace rverom

using namespace rverom;

extern "C" int rve_rom_mmax(rverom_t h, int32_t *mmax) {
    if (!h || !mmax) return RVEROM_ERR_ARG;
    int v = 0;
    for (int t = 0; t < h->n_types; ++t) v = h->types[t].m > v ? h->types[t].m : v;
    *mmax = v;
    return RVEROM_OK;
}

extern "C" int rve_rom_eval_batch_j2(rverom_t h, int64_t n_points, const int32_t *type, const double *Fbar,
                                     double *q, double *s, double *S, double *Uprev, const double *hist_in,
                                     double *hist_out, const double *plastic, double *Pbar, double *dPdF,
                                     double *rnorm, int32_t *status, void *stream) {
    if (!h || n_points < 0 || n_points > INT32_MAX) return RVEROM_ERR_ARG;
    if (h->dim != 2) return RVEROM_ERR_UNSUPPORTED;
    if (n_points == 0) return RVEROM_OK;
    if (!Fbar || !q || !s || !S || !Uprev || !hist_in || !hist_out || !plastic || !Pbar || !dPdF || !rnorm ||
        !status || hist_in == hist_out)
        return RVEROM_ERR_ARG;
    for (int t = 0; t < h->n_types; ++t)
        if (h->types[t].n > 32) return RVEROM_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = prepare_buckets(h, n_points, type, status, rnorm, st);
    if (rc != RVEROM_OK) return rc;
    int32_t mmax = 0;
    rve_rom_mmax(h, &mmax);
    for (int t = 0; t < h->n_types; ++t) {
        if (!type && t > 0) break;
        EvalArgs a = {};
        a.t = h->types[t];
        a.n_points = n_points;
        a.nmax = h->nmax;
        a.V0 = h->V0;
        a.Fbar = Fbar;
        a.q = q;
        a.s = s;
        a.S = S;
        a.Uprev = Uprev;
        a.Pbar = Pbar;
        a.dPdF = dPdF;
        a.rnorm = rnorm;
        a.status = status;
        if (type) {
            a.perm = h->perm;
            a.count = h->bucket_small + t;
            a.offset = h->bucket_small + (RVEROM_MAX_TYPES + 1) + t;
        }
        J2Args j;
        j.hist_in = hist_in;
        j.hist_out = hist_out;
        j.mmax = mmax;
        for (int ph = 0; ph < 2; ++ph) {
            const double y0 = plastic[(t * 2 + ph) * 2], hk = plastic[(t * 2 + ph) * 2 + 1];
            j.sy0[ph] = (y0 > 0.0) ? y0 : INFINITY;  // sy0 <= 0 or inf: elastic phase
            j.hk[ph] = hk;
        }
        cudaError_t e;
        const int n = a.t.n;
        if (n <= 12) e = launch_j2<16>(a, j, h->n_sm, n_points, st);
        else if (n <= 24) e = launch_j2<28>(a, j, h->n_sm, n_points, st);
        else e = launch_j2<36>(a, j, h->n_sm, n_points, st);
        if (e != cudaSuccess) return RVEROM_ERR_CUDA;
    }
    return RVEROM_OK;
}
