// rverom_macro.cu -- macro level of the FE^2 step: deformation gradient at
// the macro integration points, element residual/stiffness assembly from
// (Pbar, dPdF) (Eq. 6 of the paper and its linearization), convergence norms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/rverom.h"
#include "tc.cuh"

struct rverom_mesh_s {
    int dim = 2, nen = 4, ngp = 4;
    int64_t n_nodes = 0, n_elem = 0, n_ip = 0, n_dof = 0, nnz = 0;
    int n_sm = 1;
    int32_t *conn = nullptr;     // device [n_elem][nen]
    double *dN = nullptr;        // device [n_ip][nen][d]
    double *wJ0 = nullptr;       // device [n_ip]
    int32_t *kmap = nullptr;     // device [n_elem][(nen d)^2] CSR index of K_e entries
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    // global solve (macro_solve): device CSR pattern, CSR index of each
    // row's diagonal-block start, and the solver's workspace
    int32_t *rowp = nullptr;     // device [n_dof + 1]
    int32_t *colv = nullptr;     // device [nnz]
    int32_t *dpos = nullptr;     // device [n_dof]: index of entry (node d + i, node d) in row node d + i
    double *work = nullptr;      // device: r, u, p, s, x [n_dof] each; block inverses [n_nodes][d][d]; w [n_dof]
    double *part = nullptr;      // device [2][3][solve_blocks] per-block partial sums (double-buffered)
    unsigned *sync = nullptr;    // device [4]: grid-barrier count and generation, error flag
    int solve_blocks = 0;
};

namespace {

// isoparametric reference corners, same node order as the element connectivity
void ref_corner(int d, int a, double *s) {
    static const int c2[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    static const int c3[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                 {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
    for (int k = 0; k < d; ++k) s[k] = d == 2 ? c2[a][k] : c3[a][k];
}

bool invert(int d, const double *J, double *Ji, double &det) {
    if (d == 2) {
        det = J[0] * J[3] - J[1] * J[2];
        if (!(det > 0)) return false;
        Ji[0] = J[3] / det;
        Ji[1] = -J[1] / det;
        Ji[2] = -J[2] / det;
        Ji[3] = J[0] / det;
        return true;
    }
    det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
    if (!(det > 0)) return false;
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    return true;
}

__global__ void k_gradient(int D, int nen, int ngp, int64_t p0, int64_t n_ip, const int32_t *conn, const double *dN,
                           const double *u, double *Fbar) {
    // points p0 .. p0 + n_ip - 1, written to Fbar from its start
    const int G = D * D;
    for (int64_t pl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pl < n_ip; pl += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + pl, e = p / ngp;
        double F[9];
        for (int c = 0; c < G; ++c) F[c] = (c % (D + 1) == 0) ? 1.0 : 0.0;
        for (int a = 0; a < nen; ++a) {
            const int64_t node = conn[e * nen + a];
            for (int i = 0; i < D; ++i) {
                const double ui = u[node * D + i];
                for (int J = 0; J < D; ++J) F[i * D + J] += ui * dN[(p * nen + a) * D + J];
            }
        }
        for (int c = 0; c < G; ++c) Fbar[pl * G + c] = F[c];
    }
}

// one thread per (element, local row (a, i)): row of R_e and K_e, summed over
// the element's integration points, scattered with atomics
template <int D>
__global__ void k_assemble(int64_t e0, int64_t n_elem, const int32_t *conn, const double *dN, const double *wJ0,
                           const double *Pbar, const double *dPdF, const int32_t *kmap, double *R,
                           double *Kvals) {
    // elements e0 .. e0 + n_elem - 1; Pbar and dPdF hold their points only
    constexpr int G = D * D, NEN = 1 << D, NGP = 1 << D, ND = NEN * D;
    const int64_t total = n_elem * ND;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t el = x / ND, e = e0 + el;
        const int row = (int)(x % ND);
        const int a = row / D, i = row % D;
        double r = 0.0;
        double krow[ND];
#pragma unroll
        for (int b = 0; b < ND; ++b) krow[b] = 0.0;
        for (int gp = 0; gp < NGP; ++gp) {
            const int64_t p = e * NGP + gp, pl = el * NGP + gp;
            const double w = wJ0[p];
            const double *dn = dN + p * NEN * D;
#pragma unroll
            for (int J = 0; J < D; ++J) r += w * Pbar[pl * G + i * D + J] * dn[a * D + J];
            if (Kvals) {
                // t[kL] = w sum_J dN_a,J C[iJ][kL]
                double t[G];
#pragma unroll
                for (int c = 0; c < G; ++c) t[c] = 0.0;
#pragma unroll
                for (int J = 0; J < D; ++J) {
                    const double f = w * dn[a * D + J];
                    const double *C = dPdF + (pl * G + i * D + J) * G;
#pragma unroll
                    for (int c = 0; c < G; ++c) t[c] += f * C[c];
                }
#pragma unroll
                for (int b = 0; b < NEN; ++b)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        double v = 0.0;
#pragma unroll
                        for (int L = 0; L < D; ++L) v += t[k * D + L] * dn[b * D + L];
                        krow[b * D + k] += v;
                    }
            }
        }
        const int64_t node = conn[e * NEN + a];
        atomicAdd(&R[node * D + i], r);
        if (Kvals) {
            const int32_t *km = kmap + (e * ND + row) * ND;
#pragma unroll
            for (int b = 0; b < ND; ++b) atomicAdd(&Kvals[km[b]], krow[b]);
        }
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void k_norms(int64_t n_dof, const double *R, const uint8_t *free_mask, int64_t n_pts, const double *rnorm,
                        double *out) {
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_dof; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fabs(R[i]);
        if (free_mask[i]) m0 = fmax(m0, v);
        else m1 = fmax(m1, v);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pts; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = rnorm[i];
        m2 = (v == v) ? fmax(m2, fabs(v)) : __longlong_as_double(0x7ff0000000000000ll);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, off));
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, off));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(out + 0, m0);
        atomic_max_nonneg(out + 1, m1);
        atomic_max_nonneg(out + 2, m2);
    }
}

bool solve_setup(rverom_mesh_s *m, const std::vector<int32_t> &rowp32, const std::vector<int32_t> &dpos);

int grid_for(int64_t work, int n_sm) {
    int64_t g = (work + 255) / 256;
    if (g > 8LL * n_sm) g = 8LL * n_sm;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

extern "C" int macro_mesh_create(int32_t dim, int64_t n_nodes, int64_t n_elem, const double *X, const int64_t *conn,
                                 rverom_mesh_t *out) {
    if (!out) return RVEROM_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || n_nodes < 1 || n_elem < 1 || !X || !conn) return RVEROM_ERR_ARG;
    if (n_nodes * dim > INT32_MAX) return RVEROM_ERR_ARG;
    const int d = dim, nen = 1 << d, ngp = 1 << d, nd = nen * d;
    for (int64_t x = 0; x < n_elem * nen; ++x)
        if (conn[x] < 0 || conn[x] >= n_nodes) return RVEROM_ERR_ARG;
    rverom_mesh_s *m = new (std::nothrow) rverom_mesh_s();
    if (!m) return RVEROM_ERR_ARG;
    m->dim = d;
    m->nen = nen;
    m->ngp = ngp;
    m->n_nodes = n_nodes;
    m->n_elem = n_elem;
    m->n_ip = n_elem * ngp;
    m->n_dof = n_nodes * d;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, dev);
    // Gauss points: lexicographic with the first reference coordinate fastest
    const double g1 = 1.0 / std::sqrt(3.0);
    std::vector<double> dN((size_t)m->n_ip * nen * d), wJ0((size_t)m->n_ip);
    for (int64_t e = 0; e < n_elem; ++e) {
        for (int gp = 0; gp < ngp; ++gp) {
            double xi[3];
            for (int k = 0; k < d; ++k) xi[k] = ((gp >> k) & 1) ? g1 : -g1;
            double dNdxi[8][3];
            for (int a = 0; a < nen; ++a) {
                double s[3];
                ref_corner(d, a, s);
                for (int k = 0; k < d; ++k) {
                    double v = s[k] / 2.0;
                    for (int l = 0; l < d; ++l)
                        if (l != k) v *= (1.0 + xi[l] * s[l]) / 2.0;
                    dNdxi[a][k] = v;
                }
            }
            double Jm[9] = {0}, Ji[9], det = 0;
            for (int a = 0; a < nen; ++a) {
                const int64_t node = conn[e * nen + a];
                for (int I = 0; I < d; ++I)
                    for (int k = 0; k < d; ++k) Jm[I * d + k] += X[node * d + I] * dNdxi[a][k];
            }
            if (!invert(d, Jm, Ji, det)) {
                delete m;
                return RVEROM_ERR_ARG;
            }
            const int64_t p = e * ngp + gp;
            wJ0[p] = det;
            for (int a = 0; a < nen; ++a)
                for (int I = 0; I < d; ++I) {
                    double v = 0.0;
                    for (int k = 0; k < d; ++k) v += dNdxi[a][k] * Ji[k * d + I];
                    dN[((size_t)p * nen + a) * d + I] = v;
                }
        }
    }
    // CSR pattern over DOFs node*d + i: all pairs of nodes sharing an element
    std::vector<std::vector<int32_t>> adj((size_t)n_nodes);
    for (int64_t e = 0; e < n_elem; ++e)
        for (int a = 0; a < nen; ++a)
            for (int b = 0; b < nen; ++b) adj[conn[e * nen + a]].push_back((int32_t)conn[e * nen + b]);
    for (auto &v : adj) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    m->row_ptr.assign((size_t)m->n_dof + 1, 0);
    for (int64_t node = 0; node < n_nodes; ++node)
        for (int i = 0; i < d; ++i) m->row_ptr[node * d + i + 1] = (int64_t)adj[node].size() * d;
    for (int64_t r = 0; r < m->n_dof; ++r) m->row_ptr[r + 1] += m->row_ptr[r];
    m->nnz = m->row_ptr[m->n_dof];
    m->col.resize((size_t)m->nnz);
    for (int64_t node = 0; node < n_nodes; ++node)
        for (int i = 0; i < d; ++i) {
            int64_t o = m->row_ptr[node * d + i];
            for (int32_t nb : adj[node])
                for (int k = 0; k < d; ++k) m->col[o++] = nb * d + k;
        }
    std::vector<int32_t> kmap((size_t)n_elem * nd * nd);
    for (int64_t e = 0; e < n_elem; ++e)
        for (int a = 0; a < nen; ++a)
            for (int i = 0; i < d; ++i) {
                const int64_t node = conn[e * nen + a];
                const auto &nb = adj[node];
                for (int b = 0; b < nen; ++b) {
                    const int32_t nodeb = (int32_t)conn[e * nen + b];
                    const int64_t pos = std::lower_bound(nb.begin(), nb.end(), nodeb) - nb.begin();
                    for (int k = 0; k < d; ++k)
                        kmap[((size_t)e * nd + a * d + i) * nd + b * d + k] =
                            (int32_t)(m->row_ptr[node * d + i] + pos * d + k);
                }
            }
    if (m->nnz > INT32_MAX) {
        delete m;
        return RVEROM_ERR_ARG;
    }
    std::vector<int32_t> rowp32((size_t)m->n_dof + 1), dpos((size_t)m->n_dof);
    for (size_t r = 0; r <= (size_t)m->n_dof; ++r) rowp32[r] = (int32_t)m->row_ptr[r];
    for (int64_t node = 0; node < n_nodes; ++node) {
        const auto &nb = adj[node];
        const int64_t pos = std::lower_bound(nb.begin(), nb.end(), (int32_t)node) - nb.begin();
        for (int i = 0; i < d; ++i) dpos[node * d + i] = (int32_t)(m->row_ptr[node * d + i] + pos * d);
    }
    std::vector<int32_t> conn32((size_t)n_elem * nen);
    for (size_t x = 0; x < conn32.size(); ++x) conn32[x] = (int32_t)conn[x];
    bool ok = cudaMalloc(&m->conn, conn32.size() * 4) == cudaSuccess &&
              cudaMalloc(&m->dN, dN.size() * 8) == cudaSuccess && cudaMalloc(&m->wJ0, wJ0.size() * 8) == cudaSuccess &&
              cudaMalloc(&m->kmap, kmap.size() * 4) == cudaSuccess &&
              cudaMemcpy(m->conn, conn32.data(), conn32.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(m->dN, dN.data(), dN.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(m->wJ0, wJ0.data(), wJ0.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(m->kmap, kmap.data(), kmap.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && solve_setup(m, rowp32, dpos);
    if (!ok) {
        macro_mesh_destroy(m);
        return RVEROM_ERR_CUDA;
    }
    *out = m;
    return RVEROM_OK;
}

extern "C" int macro_mesh_destroy(rverom_mesh_t m) {
    if (!m) return RVEROM_ERR_ARG;
    cudaDeviceSynchronize();
    cudaFree(m->conn);
    cudaFree(m->dN);
    cudaFree(m->wJ0);
    cudaFree(m->kmap);
    cudaFree(m->rowp);
    cudaFree(m->colv);
    cudaFree(m->dpos);
    cudaFree(m->work);
    cudaFree(m->part);
    cudaFree(m->sync);
    delete m;
    return RVEROM_OK;
}

extern "C" int macro_mesh_sizes(rverom_mesh_t m, int64_t *n_ip, int64_t *n_dof, int64_t *nnz) {
    if (!m) return RVEROM_ERR_ARG;
    if (n_ip) *n_ip = m->n_ip;
    if (n_dof) *n_dof = m->n_dof;
    if (nnz) *nnz = m->nnz;
    return RVEROM_OK;
}

extern "C" int macro_mesh_csr(rverom_mesh_t m, int64_t *row_ptr, int32_t *col) {
    if (!m || !row_ptr || !col) return RVEROM_ERR_ARG;
    std::copy(m->row_ptr.begin(), m->row_ptr.end(), row_ptr);
    std::copy(m->col.begin(), m->col.end(), col);
    return RVEROM_OK;
}

extern "C" int macro_gradient(rverom_mesh_t m, const double *u, double *Fbar, void *stream) {
    if (!m || !u || !Fbar) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    k_gradient<<<grid_for(m->n_ip, m->n_sm), 256, 0, st>>>(m->dim, m->nen, m->ngp, 0, m->n_ip, m->conn, m->dN, u,
                                                           Fbar);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

extern "C" int macro_gradient_range(rverom_mesh_t m, int64_t e_begin, int64_t e_end, const double *u, double *Fbar,
                                    void *stream) {
    if (!m || !u || (!Fbar && e_end > e_begin)) return RVEROM_ERR_ARG;
    if (e_begin < 0 || e_end < e_begin || e_end > m->n_elem) return RVEROM_ERR_ARG;
    if (e_end == e_begin) return RVEROM_OK;
    const int64_t n = (e_end - e_begin) * m->ngp;
    k_gradient<<<grid_for(n, m->n_sm), 256, 0, (cudaStream_t)stream>>>(m->dim, m->nen, m->ngp, e_begin * m->ngp, n,
                                                                       m->conn, m->dN, u, Fbar);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

static int launch_assemble(rverom_mesh_t m, int64_t e0, int64_t n_elem, const double *Pbar, const double *dPdF,
                           double *R, double *Kvals, cudaStream_t st) {
    const int64_t work = n_elem * m->nen * m->dim;
    if (m->dim == 2)
        k_assemble<2><<<grid_for(work, m->n_sm), 256, 0, st>>>(e0, n_elem, m->conn, m->dN, m->wJ0, Pbar, dPdF,
                                                               m->kmap, R, Kvals);
    else
        k_assemble<3><<<grid_for(work, m->n_sm), 256, 0, st>>>(e0, n_elem, m->conn, m->dN, m->wJ0, Pbar, dPdF,
                                                               m->kmap, R, Kvals);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

extern "C" int macro_assemble(rverom_mesh_t m, const double *Pbar, const double *dPdF, double *R, double *Kvals,
                              void *stream) {
    if (!m || !Pbar || !R) return RVEROM_ERR_ARG;
    if (Kvals && !dPdF) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), st) != cudaSuccess) return RVEROM_ERR_CUDA;
    if (Kvals && cudaMemsetAsync(Kvals, 0, m->nnz * sizeof(double), st) != cudaSuccess) return RVEROM_ERR_CUDA;
    return launch_assemble(m, 0, m->n_elem, Pbar, dPdF, R, Kvals, st);
}

extern "C" int macro_assemble_range(rverom_mesh_t m, int64_t e_begin, int64_t e_end, const double *Pbar,
                                    const double *dPdF, double *R, double *Kvals, void *stream) {
    if (!m || !R) return RVEROM_ERR_ARG;
    if (e_begin < 0 || e_end < e_begin || e_end > m->n_elem) return RVEROM_ERR_ARG;
    if (e_end == e_begin) return RVEROM_OK;
    if (!Pbar || (Kvals && !dPdF)) return RVEROM_ERR_ARG;
    return launch_assemble(m, e_begin, e_end - e_begin, Pbar, dPdF, R, Kvals, (cudaStream_t)stream);
}

extern "C" int macro_residual_norms(rverom_mesh_t m, const double *R, const uint8_t *free_mask, int64_t n_points,
                                    const double *rnorm, double *out, void *stream) {
    if (!m || !R || !free_mask || !out || n_points < 0 || (n_points > 0 && !rnorm)) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(out, 0, 3 * sizeof(double), st) != cudaSuccess) return RVEROM_ERR_CUDA;
    const int64_t work = m->n_dof > n_points ? m->n_dof : n_points;
    k_norms<<<grid_for(work, m->n_sm), 256, 0, st>>>(m->n_dof, R, free_mask, n_points, rnorm, out);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Global macro solve: K du = -R on the free DOFs (du = 0 on the prescribed
// ones), the Newton correction of the monolithic scheme (Sec. 2, Eq. 6 and
// its linearization; the paper solves it with a direct solver).  Conjugate
// gradients preconditioned by the inverse nodal d x d diagonal blocks of K,
// in one persistent cooperative kernel (one block per SM): every block owns a
// slice of the nodes and rows; per iteration, two grid barriers separate the
// node-wise update from the sparse product and the sparse product from the
// combined reduction.  Dot products are reduced per block and summed by every
// block in the same order, so that all blocks take the same decisions.
namespace {

constexpr int SOLVE_THREADS = 256;

struct SolveArgs {
    int64_t n_nodes, n_dof;
    const int32_t *rowp, *col, *dpos;
    const double *K, *R;
    const uint8_t *free_mask;
    double *u, *du, *info;
    double tol;
    int max_iter;
    double *r, *z, *p, *q, *x, *minv, *part;
    unsigned *sync;
};

// grid barrier with a bounded wait: false (and the error flag set) once any
// block's wait has run out
__device__ bool grid_barrier(unsigned *sync, unsigned nblk) {
    __shared__ unsigned s_ok;  // one reading per block, so that all its threads agree
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = sync + 1;
        volatile unsigned *verr = sync + 2;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(sync, 1u) == nblk - 1) {
            atomicExch(sync, 0u);
            __threadfence();
            atomicAdd(sync + 1, 1u);
        } else {
            const uint64_t t0 = rverom::tc::globaltimer_ns();
            while (*vgen == g && *verr == 0) {
                if (rverom::tc::globaltimer_ns() - t0 > rverom::tc::WAIT_LIMIT_NS) {
                    atomicExch(sync + 2, 1u);
                    break;
                }
            }
        }
        __threadfence();
        s_ok = *verr == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// sum of this block's values v over its threads (every thread gets the sum)
__device__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < SOLVE_THREADS / 32; ++k) t += sh[k];
    return t;
}

// sums over this block's threads of NV values each, in one shared-memory
// round (every thread gets the sums; sh holds 8 NV doubles)
template <int NV>
__device__ void block_sums(double (&v)[NV], double *sh) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[8 * k + w] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < SOLVE_THREADS / 32; ++j) t += sh[8 * k + j];
        v[k] = t;
    }
}

// sums of the per-block partials of NV quantities (written by other blocks:
// read past L1), one partial per thread and the same order in every block
template <int NV>
__device__ void grid_sums(const double *part, unsigned nblk, double *sh, double (&out)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = threadIdx.x < nblk ? __ldcg(part + k * nblk + threadIdx.x) : 0.0;
    block_sums<NV>(out, sh);
}

template <int D>
__device__ __forceinline__ void apply_minv(const double *minv, int64_t nd, const double (&rv)[D], const uint8_t *fm,
                                           double (&zv)[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        double zi = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) zi += minv[nd * D * D + i * D + k] * rv[k];
        zv[i] = fm[nd * D + i] ? zi : 0.0;
    }
}

// Preconditioned conjugate gradients in the single-reduction form of
// Chronopoulos and Gear: per iteration one sparse product w = K u and one
// combined reduction of (r, u), (w, u), (r, r), so two grid barriers.
template <int D>
__global__ void __launch_bounds__(SOLVE_THREADS) k_pcg(SolveArgs a) {
    __shared__ double sh[32];
    const unsigned nblk = gridDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)nblk * blockDim.x;
    double *s_ = a.q;  // s = K p
    double *wv = a.minv + a.n_nodes * D * D;  // w = K u  [n_dof]
    constexpr int LPR = D == 2 ? 8 : 16;       // lanes per row of the sparse product
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    // sparse product w = K u on the free rows (u vanishes on the prescribed
    // DOFs) with the partial (w, u); a warp takes RPW consecutive rows
    auto spmv = [&](double &wu) {
        for (int64_t r0 = (tid >> 5) * RPW; r0 < a.n_dof; r0 += (nth >> 5) * RPW) {
            const int64_t row = r0 + lane / LPR;
            double v = 0.0;
            if (row < a.n_dof && a.free_mask[row]) {
                const int32_t b0 = a.rowp[row], b1 = a.rowp[row + 1];
                for (int32_t e = b0 + sub; e < b1; e += LPR) v += a.K[e] * __ldcg(a.z + a.col[e]);
            }
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, LPR);
            if (sub == 0 && row < a.n_dof) {
                wv[row] = v;
                wu += v * __ldcg(a.z + row);
            }
        }
    };
    // preconditioner: inverse of each node's diagonal block with the rows and
    // columns of prescribed DOFs replaced by the identity; b = -R on the free
    // DOFs; x = 0, r = b, u = M r (stored in z), p = s = 0
    double bb = 0.0, ru = 0.0;
    for (int64_t nd = tid; nd < a.n_nodes; nd += nth) {
        double Bk[D * D], Bi[D * D];
        bool fr[D];
#pragma unroll
        for (int i = 0; i < D; ++i) fr[i] = a.free_mask[nd * D + i] != 0;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k)
                Bk[i * D + k] = (fr[i] && fr[k]) ? a.K[a.dpos[nd * D + i] + k] : (i == k ? 1.0 : 0.0);
        double det;
        if (D == 2) {
            det = Bk[0] * Bk[3] - Bk[1] * Bk[2];
            Bi[0] = Bk[3] / det;
            Bi[1] = -Bk[1] / det;
            Bi[2] = -Bk[2] / det;
            Bi[3] = Bk[0] / det;
        } else {
            det = Bk[0] * (Bk[4] * Bk[8] - Bk[5] * Bk[7]) - Bk[1] * (Bk[3] * Bk[8] - Bk[5] * Bk[6]) +
                  Bk[2] * (Bk[3] * Bk[7] - Bk[4] * Bk[6]);
            Bi[0] = (Bk[4] * Bk[8] - Bk[5] * Bk[7]) / det;
            Bi[1] = (Bk[2] * Bk[7] - Bk[1] * Bk[8]) / det;
            Bi[2] = (Bk[1] * Bk[5] - Bk[2] * Bk[4]) / det;
            Bi[3] = (Bk[5] * Bk[6] - Bk[3] * Bk[8]) / det;
            Bi[4] = (Bk[0] * Bk[8] - Bk[2] * Bk[6]) / det;
            Bi[5] = (Bk[2] * Bk[3] - Bk[0] * Bk[5]) / det;
            Bi[6] = (Bk[3] * Bk[7] - Bk[4] * Bk[6]) / det;
            Bi[7] = (Bk[1] * Bk[6] - Bk[0] * Bk[7]) / det;
            Bi[8] = (Bk[0] * Bk[4] - Bk[1] * Bk[3]) / det;
        }
        if (!(det > 0.0) || !isfinite(det)) {  // not positive definite: no scaling of this node
#pragma unroll
            for (int c = 0; c < D * D; ++c) Bi[c] = (c % (D + 1) == 0) ? 1.0 : 0.0;
        }
#pragma unroll
        for (int c = 0; c < D * D; ++c) a.minv[nd * D * D + c] = Bi[c];
        double rv[D], uv[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            rv[i] = fr[i] ? -a.R[nd * D + i] : 0.0;
            bb += rv[i] * rv[i];
        }
        apply_minv<D>(a.minv, nd, rv, a.free_mask, uv);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int64_t k = nd * D + i;
            a.r[k] = rv[i];
            a.z[k] = uv[i];
            a.p[k] = 0.0;
            s_[k] = 0.0;
            a.x[k] = 0.0;
            ru += rv[i] * uv[i];
        }
    }
    bool ok = grid_barrier(a.sync, nblk);  // u complete
    double wu = 0.0;
    if (ok) spmv(wu);
    {
        const double b1 = block_sum(bb, sh), b2 = block_sum(ru, sh + 8), b3 = block_sum(wu, sh + 16);
        if (threadIdx.x == 0) {
            a.part[blockIdx.x] = b2;             // (r, u)
            a.part[nblk + blockIdx.x] = b3;      // (w, u)
            a.part[2 * nblk + blockIdx.x] = b1;  // (r, r)
        }
    }
    ok = ok && grid_barrier(a.sync, nblk);
    double sums[3] = {0.0, 0.0, 0.0};
    if (ok) grid_sums<3>(a.part, nblk, sh, sums);
    double gam = sums[0], del = sums[1];
    bb = sums[2];
    double rr = bb, alpha = gam / del, beta = 0.0;
    int it = 0, status = 1;  // 1: not converged within max_iter
    const double tol2 = a.tol * a.tol * bb;
    while (ok) {
        if (rr <= tol2) {
            status = 0;
            break;
        }
        if (it >= a.max_iter) break;
        if (!(del > 0.0) || !(gam > 0.0) || !isfinite(alpha) || !(alpha > 0.0)) {  // K not positive definite
            status = 2;
            break;
        }
        // p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M r
        double pr = 0.0, prr = 0.0;
        for (int64_t nd = tid; nd < a.n_nodes; nd += nth) {
            double rv[D], uv[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const int64_t k = nd * D + i;
                const double pk = a.z[k] + beta * a.p[k];
                const double sk = __ldcg(wv + k) + beta * s_[k];
                a.p[k] = pk;
                s_[k] = sk;
                a.x[k] += alpha * pk;
                rv[i] = a.r[k] - alpha * sk;
                a.r[k] = rv[i];
                prr += rv[i] * rv[i];
            }
            apply_minv<D>(a.minv, nd, rv, a.free_mask, uv);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                a.z[nd * D + i] = uv[i];
                pr += rv[i] * uv[i];
            }
        }
        double *pt = a.part + (size_t)((it + 1) & 1) * 3 * nblk;  // partials of this iteration (double-buffered)
        {
            double v2[2] = {pr, prr};
            block_sums<2>(v2, sh);
            if (threadIdx.x == 0) {
                pt[blockIdx.x] = v2[0];
                pt[2 * nblk + blockIdx.x] = v2[1];
            }
        }
        if (!(ok = grid_barrier(a.sync, nblk))) break;  // u complete
        double pwu = 0.0;
        spmv(pwu);
        pwu = block_sum(pwu, sh + 16);
        if (threadIdx.x == 0) pt[nblk + blockIdx.x] = pwu;
        if (!(ok = grid_barrier(a.sync, nblk))) break;  // partials complete
        grid_sums<3>(pt, nblk, sh, sums);
        ++it;
        rr = sums[2];
        const double gn = sums[0];
        del = sums[1];
        beta = gn / gam;
        gam = gn;
        alpha = gn / (del - beta * gn / alpha);
    }
    if (!ok) status = 5;
    // outputs: du = x, u += x (each node by the thread that updated its x)
    for (int64_t nd = tid; nd < a.n_nodes; nd += nth)
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int64_t k = nd * D + i;
            const double v = a.x[k];
            a.du[k] = v;
            if (a.u) a.u[k] += v;
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.info[0] = (double)it;
        a.info[1] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        a.info[2] = (double)status;
    }
}

bool solve_setup(rverom_mesh_s *m, const std::vector<int32_t> &rowp32, const std::vector<int32_t> &dpos) {
    const int d = m->dim;
    int occ = 0;
    cudaError_t e = m->dim == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg<2>, SOLVE_THREADS, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg<3>, SOLVE_THREADS, 0);
    if (e != cudaSuccess || occ < 1) return false;
    // one block per SM (an iteration is latency-bound; on the 16 384-point
    // plate 152 blocks took 18 us per iteration, 37 blocks 27 us), at most
    // SOLVE_THREADS (one partial per thread in grid_sums)
    m->solve_blocks = m->n_sm < SOLVE_THREADS ? m->n_sm : SOLVE_THREADS;
    const size_t nw = (size_t)m->n_dof * 6 + (size_t)m->n_nodes * d * d;
    return cudaMalloc(&m->rowp, rowp32.size() * 4) == cudaSuccess &&
           cudaMalloc(&m->colv, m->col.size() * 4) == cudaSuccess &&
           cudaMalloc(&m->dpos, dpos.size() * 4) == cudaSuccess && cudaMalloc(&m->work, nw * 8) == cudaSuccess &&
           cudaMalloc(&m->part, (size_t)6 * m->solve_blocks * 8) == cudaSuccess &&
           cudaMalloc(&m->sync, 4 * sizeof(unsigned)) == cudaSuccess &&
           cudaMemcpy(m->rowp, rowp32.data(), rowp32.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(m->colv, m->col.data(), m->col.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(m->dpos, dpos.data(), dpos.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
}

}  // namespace

extern "C" int macro_solve(rverom_mesh_t m, const double *Kvals, const double *R, const uint8_t *free_mask,
                           double tol, int32_t max_iter, double *u, double *du, double *info, void *stream) {
    if (!m || !Kvals || !R || !free_mask || !du || !info || !(tol >= 0.0) || max_iter < 0) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(m->sync, 0, 4 * sizeof(unsigned), st) != cudaSuccess) return RVEROM_ERR_CUDA;
    SolveArgs a;
    a.n_nodes = m->n_nodes;
    a.n_dof = m->n_dof;
    a.rowp = m->rowp;
    a.col = m->colv;
    a.dpos = m->dpos;
    a.K = Kvals;
    a.R = R;
    a.free_mask = free_mask;
    a.u = u;
    a.du = du;
    a.info = info;
    a.tol = tol;
    a.max_iter = max_iter;
    a.r = m->work;
    a.z = a.r + m->n_dof;
    a.p = a.z + m->n_dof;
    a.q = a.p + m->n_dof;
    a.x = a.q + m->n_dof;
    a.minv = a.x + m->n_dof;
    a.part = m->part;
    a.sync = m->sync;
    // cooperative launch: every block is resident, so the grid barriers are
    // safe (and bounded in time all the same)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)m->solve_blocks);
    cfg.blockDim = dim3(SOLVE_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = m->dim == 2 ? cudaLaunchKernelEx(&cfg, k_pcg<2>, a) : cudaLaunchKernelEx(&cfg, k_pcg<3>, a);
    return e == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}
