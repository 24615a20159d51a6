// rverom_offline.cu -- the offline (training) stage of the hyper-ROM on the
// GPU, planar RVEs (Sec. 3.2.1, 3.3):
//   rve_snapshots          full-order periodic RVE solutions along training
//                          stretch paths (the snapshots of Eq.
//                          snapshots_displacement), or the linearized
//                          responses to the unit macro strains (the elastic
//                          modes of Eq. SVD_displacement)
//   rve_mode_gradients     gradients of the modes at every micro integration
//                          point (the table of a fully integrated ROM)
//   pod_modes              POD with the elastic/inelastic split
//   ecm_training_matrix    the ECM training matrix x_f of Sec. 3.3
//   ecm_select             the leading right singular vectors of x_f
//                          (randomized subspace iteration) and the greedy
//                          non-negative point selection of Box 1
//
// RVE: the unit cell meshed by n x n bilinear quadrilaterals, 2 x 2 Gauss
// points, periodic fluctuation w (node index mod n), node 0 fixed; element
// e = ix + n iy, node v = ix + n iy; DOF v d + i, reduced numbering without
// node 0.  Micro law: the compressible Neo-Hooke law of the online path.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/rverom.h"
#include "rom_core.cuh"
#include "tc.cuh"

namespace rverom {
namespace {

constexpr int OT = 512;  // threads of the one-CTA-per-problem kernels

struct Rve2 {
    int n;                    // elements per side
    double dN[4][4][2];       // shape gradients [gauss point][corner][J]
    double wgp;               // Gauss weight (physical)
    double mu[2], kappa[2];   // per phase
};

__host__ Rve2 make_rve2(int n, const double *moduli) {
    Rve2 r;
    r.n = n;
    const double h = 1.0 / n, g1 = 1.0 / std::sqrt(3.0);
    const int cx[4] = {0, 1, 1, 0}, cy[4] = {0, 0, 1, 1};
    for (int q = 0; q < 4; ++q) {
        // Gauss points in the order of the product (xi_0, xi_1), last fastest
        const double xi[2] = {(q & 2) ? g1 : -g1, (q & 1) ? g1 : -g1};
        for (int a = 0; a < 4; ++a) {
            const double s[2] = {2.0 * cx[a] - 1.0, 2.0 * cy[a] - 1.0};
            for (int k = 0; k < 2; ++k) {
                const int o = 1 - k;
                r.dN[q][a][k] = s[k] / 2.0 * (1.0 + xi[o] * s[o]) / 2.0 * (2.0 / h);
            }
        }
    }
    r.wgp = (h / 2.0) * (h / 2.0);
    for (int p = 0; p < 2; ++p) {
        r.mu[p] = moduli[2 * p];
        r.kappa[p] = moduli[2 * p + 1];
    }
    return r;
}

__device__ __forceinline__ int corner_node(int n, int e, int a) {
    const int cx = (a == 1 || a == 2) ? 1 : 0, cy = (a >= 2) ? 1 : 0;
    const int ix = e % n, iy = e / n;
    return ((ix + cx) % n) + n * ((iy + cy) % n);
}

// block-wide sum (every thread gets it); sh has OT/32 doubles
__device__ double bsum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < OT / 32; ++k) t += sh[k];
    return t;
}
__device__ double bmax(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < OT / 32; ++k) t = fmax(t, sh[k]);
    return t;
}

// per-IP stress and weighted tangent at F = Fbar + grad w; t <- w_p P_p,
// A <- w_p A_p; false if some det F <= 0
__device__ bool rve_law(const Rve2 &g, const int32_t *phase, const double *Fbar, const double *w, double *t,
                        double *A) {
    const int n = g.n, nip = n * n * 4;
    bool ok = true;
    for (int p = threadIdx.x; p < nip; p += blockDim.x) {
        const int e = p >> 2, q = p & 3;
        double F[4] = {Fbar[0], Fbar[1], Fbar[2], Fbar[3]};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int v = corner_node(n, e, a);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int J = 0; J < 2; ++J) F[i * 2 + J] += w[v * 2 + i] * g.dN[q][a][J];
        }
        const int ph = phase[e];
        double P[4], Fi[4], lnJ;
        if (!nh_stress<2>(F, g.mu[ph], g.kappa[ph], P, Fi, lnJ)) {
            ok = false;
            continue;
        }
        const double lam = g.kappa[ph] - (2.0 / 3.0) * g.mu[ph], c3 = g.mu[ph] - lam * lnJ;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            t[p * 4 + c] = g.wgp * P[c];
            double Ar[4];
            nh_tangent_row<2, double>(Fi, lam, c3, g.mu[ph], c, Ar);
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) A[(p * 4 + c) * 4 + e2] = g.wgp * Ar[e2];
        }
    }
    return ok;
}

// out[v] = sum over the IPs around node v of dN_a^T t_p (node 0 -> 0)
__device__ void rve_gather(const Rve2 &g, const double *t, double *out) {
    const int n = g.n, nn = n * n;
    for (int v = threadIdx.x; v < nn; v += blockDim.x) {
        double s0 = 0.0, s1 = 0.0;
        if (v != 0) {
            const int vx = v % n, vy = v / n;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int cx = (a == 1 || a == 2) ? 1 : 0, cy = (a >= 2) ? 1 : 0;
                const int e = ((vx - cx + n) % n) + n * ((vy - cy + n) % n);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double *tp = t + (e * 4 + q) * 4;
                    s0 += g.dN[q][a][0] * tp[0] + g.dN[q][a][1] * tp[1];
                    s1 += g.dN[q][a][0] * tp[2] + g.dN[q][a][1] * tp[3];
                }
            }
        }
        out[v * 2] = s0;
        out[v * 2 + 1] = s1;
    }
}

// t_p = A_p grad(x) at every IP
__device__ void rve_apply_ip(const Rve2 &g, const double *A, const double *x, double *t) {
    const int n = g.n, nip = n * n * 4;
    for (int p = threadIdx.x; p < nip; p += blockDim.x) {
        const int e = p >> 2, q = p & 3;
        double gr[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int v = corner_node(n, e, a);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int J = 0; J < 2; ++J) gr[i * 2 + J] += x[v * 2 + i] * g.dN[q][a][J];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) s += A[(p * 4 + c) * 4 + e2] * gr[e2];
            t[p * 4 + c] = s;
        }
    }
}

// inverse 2 x 2 diagonal block of K_ww at every node (node 0: identity)
__device__ void rve_block_jacobi(const Rve2 &g, const double *A, double *Minv) {
    const int n = g.n, nn = n * n;
    for (int v = threadIdx.x; v < nn; v += blockDim.x) {
        double B[4] = {0.0, 0.0, 0.0, 0.0};
        const int vx = v % n, vy = v / n;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int cx = (a == 1 || a == 2) ? 1 : 0, cy = (a >= 2) ? 1 : 0;
            const int e = ((vx - cx + n) % n) + n * ((vy - cy + n) % n);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double *Ap = A + (e * 4 + q) * 16;
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        double s = 0.0;
#pragma unroll
                        for (int J = 0; J < 2; ++J)
#pragma unroll
                            for (int L = 0; L < 2; ++L) s += g.dN[q][a][J] * Ap[(i * 2 + J) * 4 + k * 2 + L] * g.dN[q][a][L];
                        B[i * 2 + k] += s;
                    }
            }
        }
        const double det = B[0] * B[3] - B[1] * B[2];
        if (v == 0 || !(det > 0.0)) {
            Minv[v * 4] = 1.0;
            Minv[v * 4 + 1] = 0.0;
            Minv[v * 4 + 2] = 0.0;
            Minv[v * 4 + 3] = 1.0;
        } else {
            Minv[v * 4] = B[3] / det;
            Minv[v * 4 + 1] = -B[1] / det;
            Minv[v * 4 + 2] = -B[2] / det;
            Minv[v * 4 + 3] = B[0] / det;
        }
    }
}

// block-Jacobi CG on K_ww x = b (b vanishes at node 0); x overwritten;
// returns iterations (negative if not converged)
__device__ int rve_cg(const Rve2 &g, const double *A, const double *Minv, const double *b, double *x, double *r,
                      double *z, double *p, double *q, double *t, double tol, int max_it, double *sh) {
    const int nn = g.n * g.n;
    double bb = 0.0, rz = 0.0;
    for (int v = threadIdx.x; v < nn; v += blockDim.x) {
        const double r0 = b[v * 2], r1 = b[v * 2 + 1];
        x[v * 2] = 0.0;
        x[v * 2 + 1] = 0.0;
        r[v * 2] = r0;
        r[v * 2 + 1] = r1;
        const double z0 = Minv[v * 4] * r0 + Minv[v * 4 + 1] * r1, z1 = Minv[v * 4 + 2] * r0 + Minv[v * 4 + 3] * r1;
        z[v * 2] = z0;
        z[v * 2 + 1] = z1;
        p[v * 2] = z0;
        p[v * 2 + 1] = z1;
        bb += r0 * r0 + r1 * r1;
        rz += r0 * z0 + r1 * z1;
    }
    bb = bsum(bb, sh);
    rz = bsum(rz, sh);
    double rr = bb;
    int it = 0;
    while (rr > tol * tol * bb && it < max_it) {
        __syncthreads();
        rve_apply_ip(g, A, p, t);
        __syncthreads();
        rve_gather(g, t, q);
        __syncthreads();
        double pq = 0.0;
        for (int v = threadIdx.x; v < nn; v += blockDim.x) pq += p[v * 2] * q[v * 2] + p[v * 2 + 1] * q[v * 2 + 1];
        pq = bsum(pq, sh);
        if (!(pq > 0.0)) return -1;
        const double alpha = rz / pq;
        double rzn = 0.0, rrn = 0.0;
        for (int v = threadIdx.x; v < nn; v += blockDim.x) {
            x[v * 2] += alpha * p[v * 2];
            x[v * 2 + 1] += alpha * p[v * 2 + 1];
            const double r0 = r[v * 2] - alpha * q[v * 2], r1 = r[v * 2 + 1] - alpha * q[v * 2 + 1];
            r[v * 2] = r0;
            r[v * 2 + 1] = r1;
            const double z0 = Minv[v * 4] * r0 + Minv[v * 4 + 1] * r1;
            const double z1 = Minv[v * 4 + 2] * r0 + Minv[v * 4 + 3] * r1;
            z[v * 2] = z0;
            z[v * 2 + 1] = z1;
            rzn += r0 * z0 + r1 * z1;
            rrn += r0 * r0 + r1 * r1;
        }
        rzn = bsum(rzn, sh);
        rr = bsum(rrn, sh);
        const double beta = rzn / rz;
        rz = rzn;
        for (int v = threadIdx.x; v < nn; v += blockDim.x) {
            p[v * 2] = z[v * 2] + beta * p[v * 2];
            p[v * 2 + 1] = z[v * 2 + 1] + beta * p[v * 2 + 1];
        }
        ++it;
    }
    __syncthreads();
    return rr <= tol * tol * bb ? it : -it - 1;
}

struct SnapArgs {
    Rve2 geo;
    const int32_t *phase;
    const double *paths;   // [n_paths][n_steps][4] macro stretch of every step (mode 0)
    int n_steps;
    int linear;            // 1: linearized responses to the unit macro strains (CTA v: strain v)
    double tol, cg_tol;
    int max_newton, max_cg;
    double *X;             // out [n_problems * n_steps][n_dof]
    double *work;
    int64_t stride;        // doubles of workspace per CTA
    double *info;          // [n_problems][4]: Newton its, CG its, final max|f|, status (0 ok)
};

__global__ void __launch_bounds__(OT) k_rve_snapshots(SnapArgs s) {
    __shared__ double sh[OT / 32];
    const Rve2 &g = s.geo;
    const int n = g.n, nn = n * n, nd = nn * 2, nip = nn * 4;
    double *w = s.work + (int64_t)blockIdx.x * s.stride;
    double *f = w + nd, *dx = f + nd, *r = dx + nd, *z = r + nd, *p = z + nd, *q = p + nd;
    double *t = q + nd, *A = t + nip * 4, *Minv = A + nip * 16;
    for (int v = threadIdx.x; v < nd; v += blockDim.x) w[v] = 0.0;
    __syncthreads();
    int newton = 0, cg = 0, status = 0;
    double fmax_last = 0.0;
    const int steps = s.linear ? 1 : s.n_steps;
    for (int k = 0; k < steps && status == 0; ++k) {
        double Fb[4] = {1.0, 0.0, 0.0, 1.0};
        if (!s.linear)
            for (int c = 0; c < 4; ++c) Fb[c] = s.paths[((int64_t)blockIdx.x * s.n_steps + k) * 4 + c];
        if (s.linear) {
            // K_ww w = -K_wF E_v at Fbar = I, w = 0
            rve_law(g, s.phase, Fb, w, t, A);
            __syncthreads();
            int i1 = blockIdx.x == 1 ? 1 : 0, j1 = blockIdx.x == 0 ? 0 : 1;
            double E[4] = {0.0, 0.0, 0.0, 0.0};
            E[i1 * 2 + j1] = 1.0;
            E[j1 * 2 + i1] = 1.0;
            for (int pp = threadIdx.x; pp < nip; pp += blockDim.x)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    double v = 0.0;
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) v += A[(pp * 4 + c) * 4 + e2] * E[e2];
                    t[pp * 4 + c] = -v;
                }
            __syncthreads();
            rve_gather(g, t, f);
            rve_block_jacobi(g, A, Minv);
            __syncthreads();
            const int it = rve_cg(g, A, Minv, f, dx, r, z, p, q, t, s.cg_tol, s.max_cg, sh);
            if (it < 0) status = 2;
            cg += it < 0 ? -it - 1 : it;
            for (int v = threadIdx.x; v < nd; v += blockDim.x) w[v] = dx[v];
            __syncthreads();
        } else {
            for (int it = 0;; ++it) {
                const bool ok = __syncthreads_and(rve_law(g, s.phase, Fb, w, t, A));
                if (!ok) {
                    status = 1;
                    break;
                }
                __syncthreads();
                rve_gather(g, t, f);
                __syncthreads();
                double fm = 0.0;
                for (int v = threadIdx.x; v < nd; v += blockDim.x) fm = fmax(fm, fabs(f[v]));
                fm = bmax(fm, sh);
                fmax_last = fm;
                if (fm <= s.tol) break;
                if (it >= s.max_newton) {
                    status = 3;
                    break;
                }
                rve_block_jacobi(g, A, Minv);
                for (int v = threadIdx.x; v < nd; v += blockDim.x) f[v] = -f[v];
                __syncthreads();
                const int ci = rve_cg(g, A, Minv, f, dx, r, z, p, q, t, s.cg_tol, s.max_cg, sh);
                cg += ci < 0 ? -ci - 1 : ci;
                for (int v = threadIdx.x; v < nd; v += blockDim.x) w[v] += dx[v];
                ++newton;
                __syncthreads();
            }
        }
        // snapshot: the reduced fluctuation (node 0 dropped)
        double *row = s.X + ((int64_t)blockIdx.x * steps + k) * (nd - 2);
        for (int v = threadIdx.x + 2; v < nd; v += blockDim.x) row[v - 2] = w[v];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s.info[blockIdx.x * 4] = newton;
        s.info[blockIdx.x * 4 + 1] = cg;
        s.info[blockIdx.x * 4 + 2] = fmax_last;
        s.info[blockIdx.x * 4 + 3] = status;
    }
}

}  // namespace
}  // namespace rverom

using namespace rverom;

extern "C" int rve_snapshots(int32_t n, const int32_t *phase, const double *moduli, int32_t n_paths,
                             int32_t n_steps, const double *paths, int32_t linear, double tol, double cg_tol,
                             int32_t max_newton, int32_t max_cg, double *X, double *info, void *stream) {
    if (n < 2 || !phase || !moduli || !X || !info || n_paths < 1 || (!linear && (n_steps < 1 || !paths)))
        return RVEROM_ERR_ARG;
    if (linear && n_paths != 3) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    SnapArgs a;
    a.geo = make_rve2(n, moduli);
    a.phase = phase;
    a.paths = paths;
    a.n_steps = linear ? 1 : n_steps;
    a.linear = linear;
    a.tol = tol;
    a.cg_tol = cg_tol;
    a.max_newton = max_newton;
    a.max_cg = max_cg;
    a.X = X;
    a.info = info;
    const int64_t nn = (int64_t)n * n;
    a.stride = nn * 2 * 8 + nn * 4 * 4 + nn * 4 * 16 + nn * 4;
    double *work = nullptr;
    if (cudaMallocAsync(&work, (size_t)a.stride * n_paths * sizeof(double), st) != cudaSuccess) return RVEROM_ERR_CUDA;
    a.work = work;
    k_rve_snapshots<<<n_paths, OT, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(work, st);
    return e == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}
