// rverom_train.cu -- outputs for updated-Lagrangian macro codes and the
// clustered training of the hyper-ROM:
//   rve_rom_biot_cauchy     Biot stress and tangent, Cauchy stress and its
//                           approximate tangent (Sec. 3.2.2, Eqs.
//                           workconjugacy and biotstress; Appendix A)
//   surrogate_linear_eval   the linear-elastic surrogate of Box 2, step 1
//   paths_kmeans            k-means of macro deformation paths, Box 2 step 3
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/rverom.h"
#include "rom_core.cuh"

namespace rverom {
namespace {

// x <- A^-1 x for NR right-hand sides (columns of x, leading dimension NR),
// Gaussian elimination with partial pivoting on the N x N matrix A
// (overwritten); false if A is singular
template <int N, int NR>
__device__ bool small_solve(double (&A)[N][N], double (&x)[N][NR]) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int pr = k;
        double pv = fabs(A[k][k]);
#pragma unroll
        for (int i = k + 1; i < N; ++i)
            if (fabs(A[i][k]) > pv) {
                pv = fabs(A[i][k]);
                pr = i;
            }
        if (!(pv > 0.0)) return false;
        if (pr != k) {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double t = A[k][j];
                A[k][j] = A[pr][j];
                A[pr][j] = t;
            }
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const double t = x[k][j];
                x[k][j] = x[pr][j];
                x[pr][j] = t;
            }
        }
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const double f = A[i][k] / A[k][k];
#pragma unroll
            for (int j = k; j < N; ++j) A[i][j] -= f * A[k][j];
#pragma unroll
            for (int j = 0; j < NR; ++j) x[i][j] -= f * x[k][j];
        }
    }
#pragma unroll
    for (int k = N - 1; k >= 0; --k)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            double v = x[k][j];
#pragma unroll
            for (int i = k + 1; i < N; ++i) v -= A[k][i] * x[i][j];
            x[k][j] = v / A[k][k];
        }
    return true;
}

// symmetric part of a d x d matrix M in tensor (not engineering) components
template <int D>
__device__ __forceinline__ double sym_comp(const double *M, int v) {
    int i, j;
    voigt_pair(D, v, i, j);
    return 0.5 * (M[i * D + j] + M[j * D + i]);
}

// C = A^T B and C = A B (d x d)
template <int D>
__device__ __forceinline__ void mtm(const double *A, const double *B, double *C) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) v += A[k * D + i] * B[k * D + j];
            C[i * D + j] = v;
        }
}
template <int D>
__device__ __forceinline__ void mm(const double *A, const double *B, double *C) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) v += A[i * D + k] * B[k * D + j];
            C[i * D + j] = v;
        }
}

// symmetric unit tensor of Voigt component v (both shear entries 1)
template <int D>
__device__ __forceinline__ void unit_sym(int v, double *E) {
#pragma unroll
    for (int c = 0; c < D * D; ++c) E[c] = 0.0;
    int i, j;
    voigt_pair(D, v, i, j);
    E[i * D + j] = 1.0;
    E[j * D + i] = 1.0;
}

template <int D>
__global__ void k_biot_cauchy(int64_t n, const double *Fbar, const double *Pbar, const double *dPdF, double *biot,
                              double *cbiot, double *sigma, double *csigma) {
    constexpr int G = D * D, NS = Dims<D>::NS;
    const double dnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double F[G], P[G], R[G], U[G], Fi[G], M[G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            F[c] = Fbar[p * G + c];
            P[c] = Pbar[p * G + c];
        }
        bool ok = det<D>(F) > 0.0 && polar<D>(F, R, U);
        const double J = ok ? inverse<D>(F, Fi) : 1.0;
        // Biot stress T = sym(R^T P) (Eq. workconjugacy)
        double T[NS], CB[NS][NS], L[NS][NS], X[NS][NS + 1];
        mtm<D>(R, P, M);
#pragma unroll
        for (int v = 0; v < NS; ++v) T[v] = sym_comp<D>(M, v);
        // Biot tangent: dT for dU = E_w at fixed R (dF = R E_w, dR = 0)
#pragma unroll
        for (int w = 0; w < NS; ++w) {
            double E[G], dF[G], dP[G];
            unit_sym<D>(w, E);
            mm<D>(R, E, dF);
#pragma unroll
            for (int c = 0; c < G; ++c) {
                double v = 0.0;
#pragma unroll
                for (int e = 0; e < G; ++e) v += dPdF[(p * G + c) * G + e] * dF[e];
                dP[c] = v;
            }
            mtm<D>(R, dP, M);
#pragma unroll
            for (int v = 0; v < NS; ++v) CB[v][w] = sym_comp<D>(M, v);
        }
        // Eq. biotstress as a linear map on symmetric tensors:
        // L(sigma) = (J/2)(R^T sigma F^-T + F^-1 sigma R); and the stretch
        // rate of a rate of deformation, sym(R^T D F) (Appendix A)
        double Gm[NS][NS];
#pragma unroll
        for (int w = 0; w < NS; ++w) {
            double E[G], A1[G], A2[G], FiT[G];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) FiT[i * D + j] = Fi[j * D + i];
            unit_sym<D>(w, E);
            mtm<D>(R, E, A1);
            mm<D>(A1, FiT, A2);  // R^T E F^-T
            double B1[G], B2[G];
            mm<D>(Fi, E, B1);
            mm<D>(B1, R, B2);  // F^-1 E R
            double S[G];
#pragma unroll
            for (int c = 0; c < G; ++c) S[c] = 0.5 * J * (A2[c] + B2[c]);
#pragma unroll
            for (int v = 0; v < NS; ++v) L[v][w] = sym_comp<D>(S, v);
            mm<D>(A1, F, A2);  // R^T E F
#pragma unroll
            for (int v = 0; v < NS; ++v) Gm[v][w] = sym_comp<D>(A2, v);
        }
        // right-hand sides: T and the columns of C^B G
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            X[v][0] = T[v];
#pragma unroll
            for (int w = 0; w < NS; ++w) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < NS; ++k) s += CB[v][k] * Gm[k][w];
                X[v][w + 1] = s;
            }
        }
        ok = ok && small_solve<NS, NS + 1>(L, X);
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            if (biot) biot[p * NS + v] = ok ? T[v] : dnan;
            if (sigma) sigma[p * NS + v] = ok ? X[v][0] : dnan;
#pragma unroll
            for (int w = 0; w < NS; ++w) {
                if (cbiot) cbiot[(p * NS + v) * NS + w] = ok ? CB[v][w] : dnan;
                if (csigma) csigma[(p * NS + v) * NS + w] = ok ? X[v][w + 1] : dnan;
            }
        }
    }
}

template <int D>
__global__ void k_linear(int64_t n, const double *C0, const double *Fbar, double *Pbar, double *dPdF) {
    constexpr int G = D * D;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double H[G];
#pragma unroll
        for (int c = 0; c < G; ++c) H[c] = Fbar[p * G + c] - ((c % (D + 1) == 0) ? 1.0 : 0.0);
#pragma unroll
        for (int c = 0; c < G; ++c) {
            double v = 0.0;
#pragma unroll
            for (int e = 0; e < G; ++e) {
                const double ce = C0[c * G + e];
                v += ce * H[e];
                if (dPdF) dPdF[(p * G + c) * G + e] = ce;
            }
            Pbar[p * G + c] = v;
        }
    }
}

// squared Euclidean distance, coordinates summed in order without fused
// multiply-adds (the same rounding as a plain sequential loop)
__device__ __forceinline__ double sqdist(const double *x, const double *c, int dim) {
    double s = 0.0;
    for (int j = 0; j < dim; ++j) {
        const double d = __dsub_rn(x[j], c[j]);
        s = __dadd_rn(s, __dmul_rn(d, d));
    }
    return s;
}

__global__ void k_assign(int64_t n, int dim, const double *X, int k, const double *C, int32_t *labels,
                         unsigned *changed) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int best = 0;
        double bd = sqdist(X + p * dim, C, dim);
        for (int c = 1; c < k; ++c) {
            const double dd = sqdist(X + p * dim, C + (int64_t)c * dim, dim);
            if (dd < bd) {  // ties keep the lowest index
                bd = dd;
                best = c;
            }
        }
        if (labels[p] != best) {
            atomicAdd(changed, 1u);
            labels[p] = best;
        }
    }
}

// one block per (cluster, coordinate): the mean of the coordinate over the
// cluster's paths, summed in a fixed order; empty clusters keep their centre
__global__ void __launch_bounds__(256) k_update(int64_t n, int dim, const double *X, const int32_t *labels,
                                                double *C) {
    __shared__ double ss[256];
    __shared__ int sc[256];
    const int c = blockIdx.x / dim, j = blockIdx.x % dim;
    double s = 0.0;
    int cnt = 0;
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x)
        if (labels[p] == c) {
            s += X[p * dim + j];
            ++cnt;
        }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && sc[0] > 0) C[(int64_t)c * dim + j] = ss[0] / sc[0];
}

// per-block partial sums of the distance of every path to its centre
__global__ void __launch_bounds__(256) k_inertia(int64_t n, int dim, const double *X, const double *C,
                                                 const int32_t *labels, double *part) {
    __shared__ double ss[256];
    double s = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        s += sqdist(X + p * dim, C + (int64_t)labels[p] * dim, dim);
    ss[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) ss[threadIdx.x] += ss[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = ss[0];
}

int grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return g < 1 ? 1 : (int)g;
}

}  // namespace
}  // namespace rverom

using namespace rverom;

extern "C" int rve_rom_biot_cauchy(int32_t dim, int64_t n, const double *Fbar, const double *Pbar,
                                   const double *dPdF, double *biot, double *cbiot, double *sigma, double *csigma,
                                   void *stream) {
    if ((dim != 2 && dim != 3) || n < 0) return RVEROM_ERR_ARG;
    if (n == 0) return RVEROM_OK;
    if (!Fbar || !Pbar || !dPdF) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (dim == 2) k_biot_cauchy<2><<<grid_of(n), 256, 0, st>>>(n, Fbar, Pbar, dPdF, biot, cbiot, sigma, csigma);
    else k_biot_cauchy<3><<<grid_of(n), 128, 0, st>>>(n, Fbar, Pbar, dPdF, biot, cbiot, sigma, csigma);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

extern "C" int surrogate_linear_eval(int32_t dim, int64_t n, const double *C0, const double *Fbar, double *Pbar,
                                     double *dPdF, void *stream) {
    if ((dim != 2 && dim != 3) || n < 0) return RVEROM_ERR_ARG;
    if (n == 0) return RVEROM_OK;
    if (!C0 || !Fbar || !Pbar) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (dim == 2) k_linear<2><<<grid_of(n), 256, 0, st>>>(n, C0, Fbar, Pbar, dPdF);
    else k_linear<3><<<grid_of(n), 256, 0, st>>>(n, C0, Fbar, Pbar, dPdF);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

extern "C" int paths_kmeans(int64_t n, int32_t dim, const double *X, int32_t k, double *centers, int32_t *labels,
                            int32_t max_iter, double *info, void *stream) {
    if (n < 1 || dim < 1 || k < 1 || k > n || max_iter < 0 || !X || !centers || !labels || !info)
        return RVEROM_ERR_ARG;
    if ((int64_t)k * dim > (1 << 30)) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned *changed = nullptr;
    double *part = nullptr;
    const int gi = grid_of(n);
    if (cudaMalloc(&changed, sizeof(unsigned)) != cudaSuccess) return RVEROM_ERR_CUDA;
    if (cudaMalloc(&part, gi * sizeof(double)) != cudaSuccess) {
        cudaFree(changed);
        return RVEROM_ERR_CUDA;
    }
    int rc = RVEROM_OK;
    int it = 0;
    // no path has a cluster yet: the first assignment changes every label
    if (cudaMemsetAsync(labels, 0xff, (size_t)n * sizeof(int32_t), st) != cudaSuccess) rc = RVEROM_ERR_CUDA;
    for (; rc == RVEROM_OK && it < max_iter; ++it) {
        unsigned h_changed = 0;
        if (cudaMemsetAsync(changed, 0, sizeof(unsigned), st) != cudaSuccess) rc = RVEROM_ERR_CUDA;
        k_assign<<<gi, 256, 0, st>>>(n, dim, X, k, centers, labels, changed);
        if (cudaMemcpyAsync(&h_changed, changed, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = RVEROM_ERR_CUDA;
        if (rc != RVEROM_OK || h_changed == 0) break;
        k_update<<<(unsigned)(k * dim), 256, 0, st>>>(n, dim, X, labels, centers);
    }
    if (rc == RVEROM_OK && it == max_iter) {  // labels of the final centres
        k_assign<<<gi, 256, 0, st>>>(n, dim, X, k, centers, labels, changed);
    }
    std::vector<double> hp(gi);
    if (rc == RVEROM_OK) {
        k_inertia<<<gi, 256, 0, st>>>(n, dim, X, centers, labels, part);
        if (cudaMemcpyAsync(hp.data(), part, gi * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = RVEROM_ERR_CUDA;
    }
    double inertia = 0.0;
    for (int b = 0; b < gi; ++b) inertia += hp[b];
    info[0] = (double)it;
    info[1] = inertia;
    cudaFree(changed);
    cudaFree(part);
    return rc;
}
