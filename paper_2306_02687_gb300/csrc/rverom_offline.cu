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

// ---- POD with the elastic/inelastic split (Eqs. SVD_displacement,
// snapshots_displacement) ------------------------------------------------------

// rows [n_rows][len] orthonormalized in place (modified Gram-Schmidt, twice)
__global__ void __launch_bounds__(OT) k_orthonormalize(int n_rows, int64_t len, double *rows) {
    __shared__ double sh[OT / 32];
    for (int k = 0; k < n_rows; ++k) {
        double *v = rows + (int64_t)k * len;
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < k; ++j) {
                const double *u = rows + (int64_t)j * len;
                double d = 0.0;
                for (int64_t x = threadIdx.x; x < len; x += blockDim.x) d += u[x] * v[x];
                d = bsum(d, sh);
                for (int64_t x = threadIdx.x; x < len; x += blockDim.x) v[x] -= d * u[x];
                __syncthreads();
            }
        double nr = 0.0;
        for (int64_t x = threadIdx.x; x < len; x += blockDim.x) nr += v[x] * v[x];
        nr = sqrt(bsum(nr, sh));
        for (int64_t x = threadIdx.x; x < len; x += blockDim.x) v[x] /= nr;
        __syncthreads();
    }
}

// Xm[s] = X[s] - sum_k <X[s], phi_k> phi_k over the n_el orthonormal rows phi
__global__ void __launch_bounds__(OT) k_project_out(int64_t len, const double *X, int n_el, const double *phi,
                                                     double *Xm) {
    __shared__ double sh[OT / 32];
    const double *x = X + (int64_t)blockIdx.x * len;
    double *y = Xm + (int64_t)blockIdx.x * len;
    double c[8];
    for (int k = 0; k < n_el && k < 8; ++k) {
        double d = 0.0;
        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) d += x[i] * phi[(int64_t)k * len + i];
        c[k] = bsum(d, sh);
    }
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        double v = x[i];
        for (int k = 0; k < n_el && k < 8; ++k) v -= c[k] * phi[(int64_t)k * len + i];
        y[i] = v;
    }
}

// Gram matrix G[a][b] = <R[a], R[b]> of n rows (one block per pair a <= b)
__global__ void __launch_bounds__(256) k_gram(int n, int64_t len, const double *R, double *G) {
    __shared__ double sh[8];
    int a = 0, rem = blockIdx.x;
    while (rem >= n - a) {
        rem -= n - a;
        ++a;
    }
    const int b = a + rem;
    double d = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) d += R[(int64_t)a * len + i] * R[(int64_t)b * len + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += sh[k];
        G[(int64_t)a * n + b] = t;
        G[(int64_t)b * n + a] = t;
    }
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations (one CTA): A
// [n][n] (global, overwritten: the eigenvalues end on its diagonal), V
// [n][n] the eigenvectors as columns; order [n] the indices by descending
// eigenvalue; ev [n] the sorted eigenvalues
__global__ void __launch_bounds__(OT) k_jacobi(int n, double *A, double *V, int *order, double *ev, int max_sweeps,
                                               double *info) {
    __shared__ double sh[OT / 32];
    __shared__ double cs[3];
    __shared__ int skip;
    for (int64_t x = threadIdx.x; x < (int64_t)n * n; x += blockDim.x) V[x] = (x / n == x % n) ? 1.0 : 0.0;
    __syncthreads();
    double total = 0.0;
    for (int64_t x = threadIdx.x; x < (int64_t)n * n; x += blockDim.x) total += A[x] * A[x];
    total = bsum(total, sh);
    int sweep = 0;
    double off = 0.0;
    for (; sweep < max_sweeps; ++sweep) {
        off = 0.0;
        for (int64_t x = threadIdx.x; x < (int64_t)n * n; x += blockDim.x)
            if (x / n != x % n) off += A[x] * A[x];
        off = bsum(off, sh);
        if (!(off > 1e-30 * total)) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (threadIdx.x == 0) {
                    const double apq = A[(int64_t)p * n + q], app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
                    skip = !(fabs(apq) > 1e-300) || fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq));
                    if (!skip) {
                        const double th = (aqq - app) / (2.0 * apq);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        const double c = 1.0 / sqrt(t * t + 1.0);
                        cs[0] = c;
                        cs[1] = t * c;
                        cs[2] = t;
                    }
                }
                __syncthreads();
                if (!skip) {
                    const double c = cs[0], s = cs[1], t = cs[2];
                    for (int k = threadIdx.x; k < n; k += blockDim.x) {
                        if (k != p && k != q) {
                            const double akp = A[(int64_t)k * n + p], akq = A[(int64_t)k * n + q];
                            const double np_ = c * akp - s * akq, nq_ = s * akp + c * akq;
                            A[(int64_t)k * n + p] = np_;
                            A[(int64_t)p * n + k] = np_;
                            A[(int64_t)k * n + q] = nq_;
                            A[(int64_t)q * n + k] = nq_;
                        }
                        const double vkp = V[(int64_t)k * n + p], vkq = V[(int64_t)k * n + q];
                        V[(int64_t)k * n + p] = c * vkp - s * vkq;
                        V[(int64_t)k * n + q] = s * vkp + c * vkq;
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        const double apq = A[(int64_t)p * n + q];
                        A[(int64_t)p * n + p] -= t * apq;
                        A[(int64_t)q * n + q] += t * apq;
                        A[(int64_t)p * n + q] = 0.0;
                        A[(int64_t)q * n + p] = 0.0;
                    }
                }
                __syncthreads();
            }
    }
    if (threadIdx.x == 0) {
        // indices by descending eigenvalue (insertion sort, ties by index)
        for (int i = 0; i < n; ++i) order[i] = i;
        for (int i = 1; i < n; ++i) {
            const int o = order[i];
            const double v = A[(int64_t)o * n + o];
            int j = i - 1;
            while (j >= 0 && A[(int64_t)order[j] * n + order[j]] < v) {
                order[j + 1] = order[j];
                --j;
            }
            order[j + 1] = o;
        }
        for (int i = 0; i < n; ++i) ev[i] = A[(int64_t)order[i] * n + order[i]];
        if (info) {
            info[0] = sweep;
            info[1] = sqrt(off / total);
        }
    }
}

// phi_k = sum_s V[s][order[k]] Xm[s] / sqrt(ev[k]) for k < n_out (rows of out)
__global__ void k_pod_combine(int n_snap, int64_t len, const double *Xm, const double *V, const int *order,
                              const double *ev, int n_out, double *out) {
    const int k = blockIdx.y;
    if (k >= n_out) return;
    const int col = order[k];
    const double sc = 1.0 / sqrt(ev[k]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < n_snap; ++s) v += V[(int64_t)s * n_snap + col] * Xm[(int64_t)s * len + i];
        out[(int64_t)k * len + i] = v * sc;
    }
}

// ---- fully integrated ROM table and the ECM training matrix (Sec. 3.3) ------

// B [n_ip][4][n_modes]: gradients of the modes (rows of Phi, reduced DOFs)
__global__ void k_mode_gradients(Rve2 g, int n_modes, const double *Phi, double *B) {
    const int n = g.n, nip = n * n * 4;
    const int64_t nd = (int64_t)2 * n * n - 2;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < (int64_t)nip * n_modes;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(x / n_modes), j = (int)(x % n_modes);
        const int e = p >> 2, q = p & 3;
        double gr[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int v = corner_node(n, e, a);
            if (v == 0) continue;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const double u = Phi[(int64_t)j * nd + v * 2 + i - 2];
#pragma unroll
                for (int J = 0; J < 2; ++J) gr[i * 2 + J] += u * g.dN[q][a][J];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) B[((int64_t)p * 4 + c) * n_modes + j] = gr[c];
    }
}

// per (snapshot s, point p): F = U_s + B_p q_s, P(F); rows of snapshot s:
// [B_p^T P (n_modes); P (4)] at column p
__global__ void k_ecm_integrands(Rve2 g, const int32_t *phase, int n_modes, const double *B, int n_snap,
                                 const double *U, const double *q, double *xf, int *bad) {
    const int nip = g.n * g.n * 4, nt = n_modes + 4;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < (int64_t)n_snap * nip;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(x / nip), p = (int)(x % nip);
        const double *Bp = B + (int64_t)p * 4 * n_modes;
        double F[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v = U[s * 4 + c];
            for (int j = 0; j < n_modes; ++j) v += Bp[c * n_modes + j] * q[(int64_t)s * n_modes + j];
            F[c] = v;
        }
        const int ph = phase[p >> 2];
        double P[4], Fi[4], lnJ;
        if (!nh_stress<2>(F, g.mu[ph], g.kappa[ph], P, Fi, lnJ)) {
            atomicExch(bad, 1);
            continue;
        }
        double *col = xf + (int64_t)s * nt * nip + p;
        for (int j = 0; j < n_modes; ++j) {
            double v = 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c) v += Bp[c * n_modes + j] * P[c];
            col[(int64_t)j * nip] = v;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) col[(int64_t)(n_modes + c) * nip] = P[c];
    }
}

// every row minus its integral (Gauss weight wgp, V0 = 1); sum of squares out
__global__ void __launch_bounds__(256) k_center_rows(int64_t len, double wgp, double *xf, double *rowsq) {
    __shared__ double sh[8];
    double *row = xf + (int64_t)blockIdx.x * len;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) s += row[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0.0;
    for (int k = 0; k < 8; ++k) tot += sh[k];
    const double mean = wgp * tot;  // integral / V0
    __syncthreads();
    double q2 = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const double v = row[i] - mean;
        row[i] = v;
        q2 += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = q2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += sh[k];
        rowsq[blockIdx.x] = t;
    }
}

__global__ void k_scale_rows(int64_t len, int nt, int n_modes, double sm, double ss, double *xf) {
    const int r = blockIdx.y;
    const double f = (r % nt) < n_modes ? sm : ss;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        xf[(int64_t)r * len + i] *= f;
}

// ---- empirical cubature: right singular vectors of x_f and Box 1 ------------

// C[M][N] = sum_k opA(i, k) opB(k, j); opA(i, k) = TA ? A[k lda + i] : A[i lda + k],
// opB(k, j) = TB ? B[j ldb + k] : B[k ldb + j]  (64 x 64 tiles, 4 x 4 per thread)
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const double *A, int64_t lda, const double *B,
                                              int64_t ldb, double *C, int64_t ldc) {
    __shared__ double As[16][65], Bs[16][65];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int x = threadIdx.x; x < 16 * 64; x += 256) {
            const int kk = x / 64, ii = x % 64;
            const int gi = i0 + ii, gk = k0 + kk, gj = j0 + ii;
            As[kk][ii] = (gi < M && gk < K) ? (TA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk]) : 0.0;
            Bs[kk][ii] = (gj < N && gk < K) ? (TB ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj]) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 16 * u];
                bb[u] = Bs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * bb[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gi = i0 + ty + 16 * u, gj = j0 + tx + 16 * v;
            if (gi < M && gj < N) C[(int64_t)gi * ldc + gj] = acc[u][v];
        }
}

template <bool TA, bool TB>
void gemm(int M, int N, int K, const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
          cudaStream_t st) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
}

// SVQB orthonormalization (Stathopoulos and Wu, SIAM J. Sci. Comput. 23,
// 2002) of the columns of M [m][k]: with the Gram matrix G = M^T M and the
// column scaling D = diag(G)^-1/2, the eigendecomposition D G D = W Theta W^T
// gives the orthonormal basis M D W Theta^-1/2 of span(M).  Directions with
// Theta_j <= 1e-15 max Theta (numerically outside span(M), e.g. beyond the
// rank of x_f) become zero columns instead of amplified rounding noise.
// k_svqb_scale: dsc_j = G_jj^-1/2 (0 for a zero column), G <- D G D
__global__ void __launch_bounds__(OT) k_svqb_scale(int k, double *G, double *dsc) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double d = G[(int64_t)j * k + j];
        dsc[j] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
    __syncthreads();
    for (int64_t x = threadIdx.x; x < (int64_t)k * k; x += blockDim.x) G[x] *= dsc[x / k] * dsc[x % k];
}

// C = D W Theta^-1/2 (k x k), Theta_j the diagonal that k_jacobi left in G,
// theta_max = ev[0] (descending)
__global__ void __launch_bounds__(OT) k_svqb_coef(int k, const double *G, const double *W, const double *ev,
                                                  const double *dsc, double *C) {
    const double tmax = ev[0];
    for (int64_t x = threadIdx.x; x < (int64_t)k * k; x += blockDim.x) {
        const int i = (int)(x / k), j = (int)(x % k);
        const double th = G[(int64_t)j * k + j];
        C[x] = (th > 1e-15 * tmax && tmax > 0.0) ? dsc[i] * W[x] / sqrt(th) : 0.0;
    }
}

// Lam [m][L-1] = Q [m][k] V[:, order[c]] (c < L - 1); norms[p] = |(Lam_p, 1)|
__global__ void k_lambda(int64_t m, int k, int L, const double *Q, const double *V, const int *order, double *Lam,
                         double *norms) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        double nr = 1.0;
        for (int c = 0; c < L - 1; ++c) {
            const int col = order[c];
            double v = 0.0;
            for (int j = 0; j < k; ++j) v += Q[p * k + j] * V[(int64_t)j * k + col];
            Lam[p * (L - 1) + c] = v;
            nr += v * v;
        }
        norms[p] = sqrt(nr);
    }
}

// greedy step 1: the available column most aligned with r (ties to the
// lowest index); per-block candidates
__global__ void __launch_bounds__(256) k_ecm_scores(int64_t m, int L, const double *Lam, const double *norms,
                                                    const uint8_t *avail, const double *r, double *bv, int *bi) {
    __shared__ double sv[256];
    __shared__ int si[256];
    double best = -INFINITY;
    int bidx = -1;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        if (!avail[p]) continue;
        double v = r[L - 1];
        for (int c = 0; c < L - 1; ++c) v += Lam[p * (L - 1) + c] * r[c];
        v /= norms[p];
        if (v > best) {  // p increases along the loop: ties keep the lower index
            best = v;
            bidx = (int)p;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const double v2 = sv[threadIdx.x + o];
            const int i2 = si[threadIdx.x + o];
            if (i2 >= 0 && (si[threadIdx.x] < 0 || v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x]))) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bv[blockIdx.x] = sv[0];
        bi[blockIdx.x] = si[0];
    }
}

struct EcmState {
    int L;               // rows of J (m~)
    int64_t m;
    const double *Lam;   // [m][L-1]
    double V0;
    int *z;              // [cap] selected points
    double *w;           // [cap] weights
    int *nz;             // device scalar: selected count
    uint8_t *avail;      // [m]
    double *r;           // [L] residual b - J_z w
    double *Jz, *Q, *R;  // scratch [L][cap], [L][cap], [cap][cap]
    double *s, *x;       // scratch [cap]
    int *act;            // scratch [cap] passive (1) / active (0) set of the NNLS
    int cap;
    double *stat;        // [4] device: last pick, negative flag, fit residual, NNLS solves
};

__device__ __forceinline__ double jcol(const EcmState &e, int p, int row) {
    return row < e.L - 1 ? e.Lam[(int64_t)p * (e.L - 1) + row] : 1.0;
}

// least squares min |J_S x - b| over the columns S (sel[c] != 0 of the
// current z) by classical Gram-Schmidt QR, twice; x written for c in S
// (zero elsewhere); false if a column is dependent
__device__ bool ecm_ls(const EcmState &e, int nz, const int *sel, double *xout, double *sh) {
    const int L = e.L;
    __shared__ int cols[1024];
    __shared__ int ncol;
    if (threadIdx.x == 0) {
        int c2 = 0;
        for (int c = 0; c < nz; ++c)
            if (sel[c]) cols[c2++] = c;
        ncol = c2;
    }
    __syncthreads();
    const int nc = ncol;
    for (int c = threadIdx.x; c < nz; c += blockDim.x) xout[c] = 0.0;
    for (int64_t x = threadIdx.x; x < (int64_t)nc * nc; x += blockDim.x) e.R[x] = 0.0;
    __syncthreads();
    for (int j = 0; j < nc; ++j) {
        double *qj = e.Q + (int64_t)j * L;
        for (int i = threadIdx.x; i < L; i += blockDim.x) qj[i] = jcol(e, e.z[cols[j]], i);
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            // coefficients against the previous columns, then the update
            for (int t = threadIdx.x; t < j; t += blockDim.x) {
                const double *qt = e.Q + (int64_t)t * L;
                double d = 0.0;
                for (int i = 0; i < L; ++i) d += qt[i] * qj[i];
                e.s[t] = d;
                e.R[(int64_t)t * nc + j] += d;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < L; i += blockDim.x) {
                double v = qj[i];
                for (int t = 0; t < j; ++t) v -= e.s[t] * e.Q[(int64_t)t * L + i];
                qj[i] = v;
            }
            __syncthreads();
        }
        double nr = 0.0;
        for (int i = threadIdx.x; i < L; i += blockDim.x) nr += qj[i] * qj[i];
        nr = sqrt(bsum(nr, sh));
        if (!(nr > 1e-14)) return false;
        for (int i = threadIdx.x; i < L; i += blockDim.x) qj[i] /= nr;
        if (threadIdx.x == 0) e.R[(int64_t)j * nc + j] = nr;
        __syncthreads();
    }
    // x = R^-1 Q^T b, b = (0, ..., 0, V0)
    if (threadIdx.x == 0) {
        for (int j = nc - 1; j >= 0; --j) {
            double v = e.Q[(int64_t)j * L + L - 1] * e.V0;
            for (int t = j + 1; t < nc; ++t) v -= e.R[(int64_t)j * nc + t] * e.s[t];
            e.s[j] = v / e.R[(int64_t)j * nc + j];
        }
        for (int j = 0; j < nc; ++j) xout[cols[j]] = e.s[j];
    }
    __syncthreads();
    return true;
}

// gradient g = J_z^T (b - J_z x) into e.s (all nz columns)
__device__ void ecm_grad(const EcmState &e, int nz, const double *x) {
    const int L = e.L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        double v = (i == L - 1) ? e.V0 : 0.0;
        for (int c = 0; c < nz; ++c) v -= jcol(e, e.z[c], i) * x[c];
        e.Jz[i] = v;  // residual, reusing the scratch
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nz; c += blockDim.x) {
        double v = 0.0;
        for (int i = 0; i < L; ++i) v += jcol(e, e.z[c], i) * e.Jz[i];
        e.s[c] = v;
    }
    __syncthreads();
}

// Box 1 steps 3-7 after a new point was appended (one CTA): least squares
// on the selected columns; if a weight is negative, the non-negative least
// squares of Lawson and Hanson instead; zero weights leave the set for good;
// r = b - J_z w
__global__ void __launch_bounds__(OT) k_ecm_update(EcmState e) {
    __shared__ double sh[OT / 32];
    __shared__ int sel[1024];
    __shared__ int neg;
    const int nz = *e.nz;
    for (int c = threadIdx.x; c < nz; c += blockDim.x) sel[c] = 1;
    __syncthreads();
    bool ok = ecm_ls(e, nz, sel, e.w, sh);
    if (threadIdx.x == 0) {
        neg = 0;
        for (int c = 0; c < nz; ++c) neg |= !(e.w[c] > 0.0);
        neg |= !ok;
        e.stat[1] = neg;
    }
    __syncthreads();
    int solves = 1;
    if (neg) {
        // Lawson-Hanson: x = 0, all columns active; move the column of the
        // largest gradient to the passive set, solve, step back to the
        // feasible region while some passive value is not positive
        for (int c = threadIdx.x; c < nz; c += blockDim.x) {
            e.x[c] = 0.0;
            sel[c] = 0;
        }
        __syncthreads();
        for (int outer = 0; outer < 3 * nz + 3; ++outer) {
            ecm_grad(e, nz, e.x);
            __shared__ int tpick;
            if (threadIdx.x == 0) {
                double gmax = 0.0;
                int t = -1;
                for (int c = 0; c < nz; ++c)
                    if (!sel[c] && e.s[c] > gmax) {
                        gmax = e.s[c];
                        t = c;
                    }
                tpick = (t >= 0 && gmax > 1e-12 * e.V0) ? t : -1;
                if (tpick >= 0) sel[tpick] = 1;
            }
            __syncthreads();
            if (tpick < 0) break;
            for (int inner = 0; inner < 3 * nz + 3; ++inner) {
                const bool lok = ecm_ls(e, nz, sel, e.w, sh);  // w: the passive-set solution
                ++solves;
                __shared__ int done;
                if (threadIdx.x == 0) {
                    done = 1;
                    double alpha = INFINITY;
                    for (int c = 0; c < nz; ++c)
                        if (sel[c] && !(e.w[c] > 0.0)) {
                            done = 0;
                            const double den = e.x[c] - e.w[c];
                            const double a = den > 0.0 ? e.x[c] / den : 0.0;
                            if (a < alpha) alpha = a;
                        }
                    if (!lok) done = 1;
                    if (!done) {
                        for (int c = 0; c < nz; ++c) {
                            if (!sel[c]) continue;
                            e.x[c] += alpha * (e.w[c] - e.x[c]);
                            if (!(e.x[c] > 1e-15 * e.V0)) {
                                e.x[c] = 0.0;
                                sel[c] = 0;
                            }
                        }
                    } else {
                        for (int c = 0; c < nz; ++c) e.x[c] = sel[c] ? e.w[c] : 0.0;
                    }
                }
                __syncthreads();
                if (done) break;
            }
        }
        for (int c = threadIdx.x; c < nz; c += blockDim.x) e.w[c] = e.x[c];
        __syncthreads();
    }
    // drop zero weights (for good: they stay unavailable), compact z and w
    if (threadIdx.x == 0) {
        int k = 0;
        for (int c = 0; c < nz; ++c)
            if (e.w[c] > 0.0) {
                e.z[k] = e.z[c];
                e.w[k] = e.w[c];
                ++k;
            }
        *e.nz = k;
        e.stat[3] += solves;
    }
    __syncthreads();
    const int nk = *e.nz;
    // r = b - J_z w and its norm
    double rr = 0.0;
    for (int i = threadIdx.x; i < e.L; i += blockDim.x) {
        double v = (i == e.L - 1) ? e.V0 : 0.0;
        for (int c = 0; c < nk; ++c) v -= jcol(e, e.z[c], i) * e.w[c];
        e.r[i] = v;
        rr += v * v;
    }
    rr = bsum(rr, sh);
    if (threadIdx.x == 0) e.stat[2] = sqrt(rr);
}

// append the picked point (from the per-block candidates)
__global__ void k_ecm_pick(int nb, const double *bv, const int *bi, EcmState e) {
    if (threadIdx.x != 0) return;
    double best = -INFINITY;
    int idx = -1;
    for (int b = 0; b < nb; ++b)
        if (bi[b] >= 0 && (idx < 0 || bv[b] > best || (bv[b] == best && bi[b] < idx))) {
            best = bv[b];
            idx = bi[b];
        }
    e.stat[0] = idx;
    if (idx < 0) return;
    const int nz = *e.nz;
    e.z[nz] = idx;
    e.w[nz] = 0.0;
    *e.nz = nz + 1;
    e.avail[idx] = 0;
}

__global__ void k_ecm_init(EcmState e) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < e.m; p += (int64_t)gridDim.x * blockDim.x)
        e.avail[p] = 1;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < e.L; i += blockDim.x) e.r[i] = (i == e.L - 1) ? e.V0 : 0.0;
        if (threadIdx.x == 0) {
            *e.nz = 0;
            for (int k = 0; k < 4; ++k) e.stat[k] = 0.0;
        }
    }
}

}  // namespace
}  // namespace rverom

using namespace rverom;

extern "C" int ecm_select(int64_t m, int32_t n_rows, const double *xf, double V0, int32_t m_target,
                          const double *Omega, int32_t k, int32_t power_its, int32_t *z, double *w,
                          int32_t *n_sel, double *info, void *stream) {
    if (m < 2 || n_rows < 1 || !xf || !(V0 > 0.0) || m_target < 2 || m_target > 1000 || m_target - 1 > k ||
        !Omega || k < 1 || k > n_rows || power_its < 0 || !z || !w || !n_sel || !info)
        return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int L = m_target, cap = m_target + 1;
    double *Y = nullptr, *Z = nullptr, *G = nullptr, *V = nullptr, *ev = nullptr, *Lam = nullptr, *nrm = nullptr;
    double *bv = nullptr, *scr = nullptr, *T = nullptr, *C = nullptr, *dsc = nullptr;
    int *order = nullptr, *bi = nullptr, *dz = nullptr, *dnz = nullptr, *act = nullptr;
    uint8_t *avail = nullptr;
    const int nb = 304;
    bool okm = cudaMallocAsync(&Y, (size_t)m * k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&Z, (size_t)n_rows * k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&G, (size_t)k * k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&V, (size_t)k * k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&ev, (size_t)k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&order, (size_t)k * 4, st) == cudaSuccess &&
               cudaMallocAsync(&T, (size_t)m * k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&C, (size_t)k * k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&dsc, (size_t)k * 8, st) == cudaSuccess &&
               cudaMallocAsync(&Lam, (size_t)m * (L - 1) * 8, st) == cudaSuccess &&
               cudaMallocAsync(&nrm, (size_t)m * 8, st) == cudaSuccess &&
               cudaMallocAsync(&avail, (size_t)m, st) == cudaSuccess &&
               cudaMallocAsync(&bv, nb * 8, st) == cudaSuccess && cudaMallocAsync(&bi, nb * 4, st) == cudaSuccess &&
               cudaMallocAsync(&dz, (size_t)cap * 4, st) == cudaSuccess &&
               cudaMallocAsync(&dnz, 4, st) == cudaSuccess &&
               cudaMallocAsync(&act, (size_t)cap * 4, st) == cudaSuccess &&
               cudaMallocAsync(&scr, ((size_t)L * cap * 2 + (size_t)cap * cap + 3 * (size_t)cap + L + 4 + cap) * 8, st) ==
                   cudaSuccess;
    int rc = okm ? RVEROM_OK : RVEROM_ERR_CUDA;
    auto orth = [&](double *M) {  // M [m][k] <- orthonormal basis of its span (SVQB, twice)
        for (int pass = 0; pass < 2; ++pass) {
            gemm<true, false>(k, k, (int)m, M, k, M, k, G, k, st);
            k_svqb_scale<<<1, OT, 0, st>>>(k, G, dsc);
            k_jacobi<<<1, OT, 0, st>>>(k, G, V, order, ev, 60, nullptr);
            k_svqb_coef<<<1, OT, 0, st>>>(k, G, V, ev, dsc, C);
            gemm<false, false>((int)m, k, k, M, k, C, k, T, k, st);
            cudaMemcpyAsync(M, T, (size_t)m * k * 8, cudaMemcpyDeviceToDevice, st);
        }
    };
    if (rc == RVEROM_OK) {
        // range of x_f^T: Y = x_f^T Omega, power iterations, orthonormal basis Q
        gemm<true, false>((int)m, k, n_rows, xf, m, Omega, k, Y, k, st);
        for (int it = 0; it < power_its; ++it) {
            orth(Y);
            gemm<false, false>(n_rows, k, (int)m, xf, m, Y, k, Z, k, st);
            gemm<true, false>((int)m, k, n_rows, xf, m, Z, k, Y, k, st);
        }
        orth(Y);
        // x_f Q, its Gram matrix and eigenvectors: the right singular vectors
        gemm<false, false>(n_rows, k, (int)m, xf, m, Y, k, Z, k, st);
        gemm<true, false>(k, k, n_rows, Z, k, Z, k, G, k, st);
        k_jacobi<<<1, OT, 0, st>>>(k, G, V, order, ev, 40, nullptr);
        k_lambda<<<(int)((m + 127) / 128), 128, 0, st>>>(m, k, L, Y, V, order, Lam, nrm);
        if (cudaGetLastError() != cudaSuccess) rc = RVEROM_ERR_CUDA;
    }
    EcmState e;
    e.L = L;
    e.m = m;
    e.Lam = Lam;
    e.V0 = V0;
    e.z = dz;
    e.w = scr;
    e.nz = dnz;
    e.avail = avail;
    e.r = scr + cap;
    e.Jz = e.r + L;
    e.Q = e.Jz + (size_t)L * cap;
    e.R = e.Q + (size_t)L * cap;
    e.s = e.R + (size_t)cap * cap;
    e.x = e.s + cap;
    e.stat = e.x + cap;
    e.act = act;
    e.cap = cap;
    int iters = 0, nz = 0;
    double stat[4] = {0, 0, 0, 0};
    if (rc == RVEROM_OK) {
        k_ecm_init<<<64, 256, 0, st>>>(e);
        // Box 1: pick, solve, drop, until m~ points or no candidate is left
        for (iters = 0; iters < 8 * m_target; ++iters) {
            k_ecm_scores<<<nb, 256, 0, st>>>(m, L, Lam, nrm, avail, e.r, bv, bi);
            k_ecm_pick<<<1, 32, 0, st>>>(nb, bv, bi, e);
            k_ecm_update<<<1, OT, 0, st>>>(e);
            if (cudaMemcpyAsync(&nz, dnz, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(stat, e.stat, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = RVEROM_ERR_CUDA;
                break;
            }
            if (stat[0] < 0 || nz >= m_target) break;
        }
    }
    if (rc == RVEROM_OK) {
        cudaMemcpyAsync(z, dz, (size_t)nz * 4, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(w, e.w, (size_t)nz * 8, cudaMemcpyDeviceToDevice, st);
        *n_sel = nz;
        info[0] = iters + 1;
        info[1] = stat[2];
        info[2] = stat[3];
        info[3] = 0.0;
    }
    for (void *ptr : {(void *)Y, (void *)Z, (void *)G, (void *)V, (void *)ev, (void *)Lam, (void *)nrm, (void *)bv,
                      (void *)scr, (void *)T, (void *)C, (void *)dsc, (void *)order, (void *)bi, (void *)dz, (void *)dnz, (void *)act,
                      (void *)avail})
        if (ptr) cudaFreeAsync(ptr, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == RVEROM_OK) rc = RVEROM_ERR_CUDA;
    return rc;
}

extern "C" int pod_modes(int64_t n_dof, int32_t n_snap, const double *X, int32_t n_el, const double *W_el,
                         int32_t n_modes, double *Phi, double *eig, double *info, void *stream) {
    if (n_dof < 1 || n_snap < 1 || n_el < 0 || n_el > 8 || n_modes < n_el || n_modes - n_el > n_snap || !X ||
        !Phi || !eig || (n_el > 0 && !W_el))
        return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *Xm = nullptr, *G = nullptr, *V = nullptr;
    int *order = nullptr;
    const size_t ns = (size_t)n_snap;
    if (cudaMallocAsync(&Xm, ns * n_dof * 8, st) != cudaSuccess) return RVEROM_ERR_CUDA;
    if (cudaMallocAsync(&G, ns * ns * 8, st) != cudaSuccess || cudaMallocAsync(&V, ns * ns * 8, st) != cudaSuccess ||
        cudaMallocAsync(&order, ns * 4, st) != cudaSuccess)
        return RVEROM_ERR_CUDA;
    // elastic modes: the orthonormalized linear responses
    if (n_el > 0) {
        cudaMemcpyAsync(Phi, W_el, (size_t)n_el * n_dof * 8, cudaMemcpyDeviceToDevice, st);
        k_orthonormalize<<<1, OT, 0, st>>>(n_el, n_dof, Phi);
    }
    // snapshots without their elastic part; leading left singular vectors
    // through the eigen-decomposition of their Gram matrix
    k_project_out<<<n_snap, OT, 0, st>>>(n_dof, X, n_el, Phi, Xm);
    k_gram<<<(unsigned)(ns * (ns + 1) / 2), 256, 0, st>>>(n_snap, n_dof, Xm, G);
    k_jacobi<<<1, OT, 0, st>>>(n_snap, G, V, order, eig, 40, info);
    if (n_modes > n_el) {
        dim3 grid((unsigned)((n_dof + 255) / 256 < 64 ? (n_dof + 255) / 256 : 64), (unsigned)(n_modes - n_el));
        k_pod_combine<<<grid, 256, 0, st>>>(n_snap, n_dof, Xm, V, order, eig, n_modes - n_el,
                                            Phi + (size_t)n_el * n_dof);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(Xm, st);
    cudaFreeAsync(G, st);
    cudaFreeAsync(V, st);
    cudaFreeAsync(order, st);
    return e == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

extern "C" int rve_mode_gradients(int32_t n, int32_t n_modes, const double *Phi, double *B, void *stream) {
    if (n < 2 || n_modes < 1 || !Phi || !B) return RVEROM_ERR_ARG;
    const double mod[4] = {1.0, 1.0, 1.0, 1.0};
    Rve2 g = make_rve2(n, mod);
    const int64_t work = (int64_t)n * n * 4 * n_modes;
    const int grid = (int)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
    k_mode_gradients<<<grid, 256, 0, (cudaStream_t)stream>>>(g, n_modes, Phi, B);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

extern "C" int ecm_training_matrix(int32_t n, const int32_t *phase, const double *moduli, int32_t n_modes,
                                   const double *B, int32_t n_snap, const double *U, const double *q, double *xf,
                                   void *stream) {
    if (n < 2 || !phase || !moduli || n_modes < 1 || !B || n_snap < 1 || !U || !q || !xf) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Rve2 g = make_rve2(n, moduli);
    const int64_t nip = (int64_t)n * n * 4;
    const int nt = n_modes + 4, rows = n_snap * nt;
    int *bad = nullptr;
    double *rowsq = nullptr;
    if (cudaMallocAsync(&bad, 4, st) != cudaSuccess || cudaMallocAsync(&rowsq, (size_t)rows * 8, st) != cudaSuccess)
        return RVEROM_ERR_CUDA;
    cudaMemsetAsync(bad, 0, 4, st);
    const int64_t work = (int64_t)n_snap * nip;
    k_ecm_integrands<<<(int)((work + 255) / 256 < 8192 ? (work + 255) / 256 : 8192), 256, 0, st>>>(
        g, phase, n_modes, B, n_snap, U, q, xf, bad);
    k_center_rows<<<rows, 256, 0, st>>>(nip, g.wgp, xf, rowsq);
    std::vector<double> rs(rows);
    int hbad = 0;
    int rc = RVEROM_OK;
    if (cudaMemcpyAsync(rs.data(), rowsq, (size_t)rows * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        rc = RVEROM_ERR_CUDA;
    if (rc == RVEROM_OK && hbad) rc = RVEROM_ERR_ARG;  // a training state folds a micro point
    if (rc == RVEROM_OK) {
        // the mode block and the stress block each to unit Frobenius norm
        double sm = 0.0, ss = 0.0;
        for (int r = 0; r < rows; ++r) ((r % nt) < n_modes ? sm : ss) += rs[r];
        dim3 grid((unsigned)((nip + 255) / 256 < 64 ? (nip + 255) / 256 : 64), (unsigned)rows);
        k_scale_rows<<<grid, 256, 0, st>>>(nip, nt, n_modes, sm > 0 ? 1.0 / std::sqrt(sm) : 1.0,
                                           ss > 0 ? 1.0 / std::sqrt(ss) : 1.0, xf);
        if (cudaGetLastError() != cudaSuccess) rc = RVEROM_ERR_CUDA;
    }
    cudaFreeAsync(bad, st);
    cudaFreeAsync(rowsq, st);
    return rc;
}

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
