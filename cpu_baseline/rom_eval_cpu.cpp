// rom_eval_cpu.cpp -- plain C++ float64 CPU baseline of the batched
// hyper-reduced RVE evaluation (steps a1-a7 of the online path of Lange,
// Huetter, Kiefer, arXiv 2306.02687, Sec. 3.2.2-3.2.3), OpenMP over macro
// points.  A timing baseline for the GPU path on the host cores: one plain
// loop per point, no blocking or vectorization beyond what the compiler does
// with -O3.  It shares no code with the CUDA library or the test oracle.
//
// Per point (row-major tensors, component c = i*d + J, g = d*d):
//   a1  Fbar = R U (2D: rotation angle atan2(F21 - F12, F11 + F22); 3D:
//       Newton iteration X <- (X + X^-T)/2 towards R), U = sym(R^T Fbar);
//       q <- q - s - S (U_voigt - U_prev)                (Sec. 3.2.3)
//   a2  F_i = U + B_i q                                  (Eq. ROM_assumption)
//   a3  compressible Neo-Hooke P_i, A_i = dP/dF          (plane strain: F33 = 1)
//   a4  r = sum w_i B_i^T P_i, V0 Pbar_U = sum w_i P_i   (Eq. ROMintforce, Eq. 2)
//   a5  K = sum B_i^T w_i A_i B_i, K_qF = sum B_i^T w_i A_i, K_FF = sum w_i A_i
//   a6  Cholesky of K; s = K^-1 r, X = K^-1 K_qF, S = X E,
//       Pbar_alg = (V0 Pbar_U - K_qF^T s) / V0, C_U = (K_FF - K_qF^T X) / V0
//   a7  Pbar = R Pbar_alg; dPbar/dFbar through the polar derivative
//       (R^T dF = Omega U + dU, Omega skew, dU symmetric).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int ST_OK = 0, ST_DETF = 1, ST_NONSPD = 2, ST_NONFINITE = 3;

inline void voigt_pair(int d, int v, int &i, int &j) {
    static const int p2[3][2] = {{0, 0}, {1, 1}, {0, 1}};
    static const int p3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    if (d == 2) {
        i = p2[v][0];
        j = p2[v][1];
    } else {
        i = p3[v][0];
        j = p3[v][1];
    }
}

double det(int d, const double *A) {
    if (d == 2) return A[0] * A[3] - A[1] * A[2];
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// inverse by the adjugate; returns the determinant
double inverse(int d, const double *A, double *Ai) {
    const double D = det(d, A);
    if (d == 2) {
        Ai[0] = A[3] / D;
        Ai[1] = -A[1] / D;
        Ai[2] = -A[2] / D;
        Ai[3] = A[0] / D;
        return D;
    }
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / D;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) / D;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / D;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) / D;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / D;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) / D;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / D;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) / D;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / D;
    return D;
}

void matmul(int d, const double *A, const double *B, double *C) {  // C = A B
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double v = 0.0;
            for (int k = 0; k < d; ++k) v += A[i * d + k] * B[k * d + j];
            C[i * d + j] = v;
        }
}

void matTmul(int d, const double *A, const double *B, double *C) {  // C = A^T B
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double v = 0.0;
            for (int k = 0; k < d; ++k) v += A[k * d + i] * B[k * d + j];
            C[i * d + j] = v;
        }
}

// polar decomposition F = R U (det F > 0)
bool polar(int d, const double *F, double *R, double *U) {
    if (d == 2) {
        const double th = std::atan2(F[2] - F[1], F[0] + F[3]);
        const double c = std::cos(th), s = std::sin(th);
        R[0] = c;
        R[1] = -s;
        R[2] = s;
        R[3] = c;
    } else {
        double X[9], Xi[9];
        std::memcpy(X, F, sizeof(X));
        bool conv = false;
        for (int it = 0; it < 60 && !conv; ++it) {
            if (!(inverse(3, X, Xi) > 0.0)) return false;
            double diff = 0.0, nrm = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double nx = 0.5 * (X[i * 3 + j] + Xi[j * 3 + i]);
                    diff = std::fmax(diff, std::fabs(nx - X[i * 3 + j]));
                    nrm = std::fmax(nrm, std::fabs(nx));
                    X[i * 3 + j] = nx;
                }
            conv = diff <= 1e-15 * nrm;
        }
        std::memcpy(R, X, sizeof(X));
    }
    double T[9];
    matTmul(d, R, F, T);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) U[i * d + j] = 0.5 * (T[i * d + j] + T[j * d + i]);
    return true;
}

// (dR, dU) of F = R U for a perturbation dF
void polar_derivative(int d, const double *R, const double *U, const double *dF, double *dR, double *dU) {
    double M[9], Om[9] = {0};
    matTmul(d, R, dF, M);  // R^T dF = Omega U + dU
    double trU = 0.0;
    for (int i = 0; i < d; ++i) trU += U[i * d + i];
    if (d == 2) {
        const double om = (M[2] - M[1]) / trU;
        Om[1] = -om;
        Om[2] = om;
    } else {
        // axial vector w of M - M^T; (tr U I - U) omega = w
        const double w[3] = {M[7] - M[5], M[2] - M[6], M[3] - M[1]};
        double Aq[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Aq[i * 3 + j] = (i == j ? trU : 0.0) - U[i * 3 + j];
        double Ai[9];
        inverse(3, Aq, Ai);
        double om[3];
        for (int i = 0; i < 3; ++i) om[i] = Ai[i * 3] * w[0] + Ai[i * 3 + 1] * w[1] + Ai[i * 3 + 2] * w[2];
        Om[1] = -om[2];
        Om[2] = om[1];
        Om[3] = om[2];
        Om[5] = -om[0];
        Om[6] = -om[1];
        Om[7] = om[0];
    }
    double OU[9];
    matmul(d, Om, U, OU);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            const double a = M[i * d + j] - OU[i * d + j], b = M[j * d + i] - OU[j * d + i];
            dU[i * d + j] = 0.5 * (a + b);
        }
    matmul(d, R, Om, dR);
}

struct Rom {
    int d, g, ns, n, m;
    const double *B, *w;
    const int *phase;
    double mu[2], lam[2], V0;
};

// steps a1-a7 of one point; returns the status
int eval_point(const Rom &rm, const double *Fbar, double *q, double *s, double *S, double *Uprev, double *Pbar,
               double *dPdF, double *rnorm) {
    const int d = rm.d, g = rm.g, ns = rm.ns, n = rm.n, m = rm.m;
    for (int c = 0; c < g; ++c)
        if (!std::isfinite(Fbar[c])) return ST_NONFINITE;
    if (!(det(d, Fbar) > 0.0)) return ST_DETF;
    double R[9], U[9];
    if (!polar(d, Fbar, R, U)) return ST_DETF;
    double Uv[6];
    for (int v = 0; v < ns; ++v) {
        int i, j;
        voigt_pair(d, v, i, j);
        Uv[v] = U[i * d + j];
    }
    std::vector<double> qn(n), r(n, 0.0), K((size_t)n * n, 0.0), KqF((size_t)n * g, 0.0), Y((size_t)g * n);
    double KFF[81] = {0}, VPU[9] = {0};
    for (int j = 0; j < n; ++j) {
        double v = q[j] - s[j];
        for (int k = 0; k < ns; ++k) v -= S[j * ns + k] * (Uv[k] - Uprev[k]);
        qn[j] = v;
    }
    for (int i = 0; i < m; ++i) {
        const double *Bi = rm.B + (size_t)i * g * n;
        double F[9], Fi[9];
        for (int c = 0; c < g; ++c) {
            double v = U[c];
            for (int j = 0; j < n; ++j) v += Bi[c * n + j] * qn[j];
            F[c] = v;
        }
        const double J = inverse(d, F, Fi);
        if (!(J > 0.0)) return ST_DETF;
        const double lnJ = std::log(J), mu = rm.mu[rm.phase[i]], lam = rm.lam[rm.phase[i]], wi = rm.w[i];
        double P[9], A[81];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) P[a * d + b] = mu * (F[a * d + b] - Fi[b * d + a]) + lam * lnJ * Fi[b * d + a];
        // A[iJ][kL] = lam Fi_Ji Fi_Lk + mu d_ik d_JL + (mu - lam lnJ) Fi_Li Fi_Jk
        for (int ii = 0; ii < d; ++ii)
            for (int JJ = 0; JJ < d; ++JJ)
                for (int kk = 0; kk < d; ++kk)
                    for (int LL = 0; LL < d; ++LL)
                        A[(ii * d + JJ) * g + kk * d + LL] = lam * Fi[JJ * d + ii] * Fi[LL * d + kk] +
                                                             ((ii == kk && JJ == LL) ? mu : 0.0) +
                                                             (mu - lam * lnJ) * Fi[LL * d + ii] * Fi[JJ * d + kk];
        for (int c = 0; c < g; ++c) {
            VPU[c] += wi * P[c];
            for (int j = 0; j < n; ++j) r[j] += Bi[c * n + j] * wi * P[c];
        }
        for (int c = 0; c < g; ++c)
            for (int e = 0; e < g; ++e) KFF[c * g + e] += wi * A[c * g + e];
        // Y = w A B_i (g x n); K += B_i^T Y; K_qF += B_i^T (w A)
        for (int c = 0; c < g; ++c)
            for (int j = 0; j < n; ++j) {
                double v = 0.0;
                for (int e = 0; e < g; ++e) v += A[c * g + e] * Bi[e * n + j];
                Y[c * n + j] = wi * v;
            }
        for (int j = 0; j < n; ++j) {
            for (int k = 0; k < n; ++k) {
                double v = 0.0;
                for (int c = 0; c < g; ++c) v += Bi[c * n + j] * Y[c * n + k];
                K[(size_t)j * n + k] += v;
            }
            for (int e = 0; e < g; ++e) {
                double v = 0.0;
                for (int c = 0; c < g; ++c) v += Bi[c * n + j] * A[c * g + e];
                KqF[(size_t)j * g + e] += wi * v;
            }
        }
    }
    for (int j = 0; j < n; ++j)
        if (!std::isfinite(r[j])) return ST_NONFINITE;
    // a6: Cholesky K = L L^T (in place, lower triangle)
    std::vector<double> L(K);
    for (int j = 0; j < n; ++j) {
        double v = L[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) v -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(v > 0.0)) return ST_NONSPD;
        const double ljj = std::sqrt(v);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = L[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    auto solve = [&](double *x) {  // x <- K^-1 x
        for (int i = 0; i < n; ++i) {
            double t = x[i];
            for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * x[k];
            x[i] = t / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double t = x[i];
            for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * x[k];
            x[i] = t / L[(size_t)i * n + i];
        }
    };
    std::vector<double> sn(r), X((size_t)n * g), col(n);
    solve(sn.data());
    for (int e = 0; e < g; ++e) {
        for (int j = 0; j < n; ++j) col[j] = KqF[(size_t)j * g + e];
        solve(col.data());
        for (int j = 0; j < n; ++j) X[(size_t)j * g + e] = col[j];
    }
    double Palg[9], CU[81];
    for (int c = 0; c < g; ++c) {
        double v = VPU[c];
        for (int j = 0; j < n; ++j) v -= KqF[(size_t)j * g + c] * sn[j];
        Palg[c] = v / rm.V0;
        for (int e = 0; e < g; ++e) {
            double t = KFF[c * g + e];
            for (int j = 0; j < n; ++j) t -= KqF[(size_t)j * g + c] * X[(size_t)j * g + e];
            CU[c * g + e] = t / rm.V0;
        }
    }
    // a7: Pbar = R Pbar_alg and its derivative through the polar split
    matmul(d, R, Palg, Pbar);
    for (int e = 0; e < g; ++e) {
        double dF[9] = {0}, dR[9], dU[9], t1[9], t2[9], CdU[9];
        dF[e] = 1.0;
        polar_derivative(d, R, U, dF, dR, dU);
        for (int c = 0; c < g; ++c) {
            double v = 0.0;
            for (int k = 0; k < g; ++k) v += CU[c * g + k] * dU[k];
            CdU[c] = v;
        }
        matmul(d, dR, Palg, t1);
        matmul(d, R, CdU, t2);
        for (int c = 0; c < g; ++c) dPdF[c * g + e] = t1[c] + t2[c];
    }
    // new state
    double rm_ = 0.0;
    for (int j = 0; j < n; ++j) {
        rm_ = std::fmax(rm_, std::fabs(r[j]));
        q[j] = qn[j];
        s[j] = sn[j];
        for (int v = 0; v < ns; ++v) {
            int i, jj;
            voigt_pair(d, v, i, jj);
            const int c1 = i * d + jj, c2 = jj * d + i;
            S[j * ns + v] = X[(size_t)j * g + c1] + (c1 != c2 ? X[(size_t)j * g + c2] : 0.0);
        }
    }
    for (int v = 0; v < ns; ++v) Uprev[v] = Uv[v];
    *rnorm = rm_;
    return ST_OK;
}

}  // namespace

// Evaluate n_points macro points of one RVE type (state arrays unpadded:
// q, s [n][n_modes], S [n][n_modes][ns], Uprev [n][ns]); nthreads OpenMP
// threads (<= 0: the OpenMP default).  Points with a non-OK status keep their
// input state and get NaN outputs.  Returns the number of threads used.
extern "C" int rom_eval_cpu(int dim, int n_modes, int n_ecm, const double *B, const double *w, const int *phase,
                            const double *moduli, double V0, int64_t n_points, const double *Fbar, double *q,
                            double *s, double *S, double *Uprev, double *Pbar, double *dPdF, double *rnorm,
                            int *status, int nthreads) {
    Rom rm;
    rm.d = dim;
    rm.g = dim * dim;
    rm.ns = dim == 2 ? 3 : 6;
    rm.n = n_modes;
    rm.m = n_ecm;
    rm.B = B;
    rm.w = w;
    rm.phase = phase;
    rm.V0 = V0;
    for (int k = 0; k < 2; ++k) {
        rm.mu[k] = moduli[2 * k];
        rm.lam[k] = moduli[2 * k + 1] - 2.0 / 3.0 * moduli[2 * k];
    }
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 8)
#endif
        for (int64_t a = 0; a < n_points; ++a) {
            const int g = rm.g, n = rm.n, ns = rm.ns;
            // the state is written only on success
            const int st = eval_point(rm, Fbar + a * g, q + a * n, s + a * n, S + a * n * ns, Uprev + a * ns,
                                      Pbar + a * g, dPdF + a * g * g, rnorm + a);
            status[a] = st;
            if (st != ST_OK) {
                for (int c = 0; c < g; ++c) Pbar[a * g + c] = NAN;
                for (int c = 0; c < g * g; ++c) dPdF[a * g * g + c] = NAN;
                rnorm[a] = NAN;
            }
        }
#ifdef _OPENMP
    }
#endif
    return used;
}
