// rverom_adjoint.cu -- implicit-function adjoint of the converged hyper-reduced
// equilibrium (rve_rom_adjoint).  The kernel is the evaluation template in
// adjoint mode: it rebuilds and condenses the reduced system at the given
// (converged) amplitudes, writes gFbar = dPdF^T gPbar, forms
// z = K^-1 K_qF R^T gPbar and accumulates, in a second pass over the ECM
// points, (1/V0) w_i <R^T gPbar - B_i z, dP_i/d(mu, kappa)> per phase.  Each
// CTA leaves its sums in the handle's partials workspace; a one-thread kernel
// adds them in block order (deterministic) into gTheta.
#include <cuda_runtime.h>

#include "../../include/rverom.h"
#include "rom_core.cuh"
#include "rverom_internal.h"

using namespace rverom;

namespace {
__global__ void k_theta_reduce(const double *partials, int nblocks, double *gTheta) {
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partials[(int64_t)b * 4 + threadIdx.x];
        gTheta[threadIdx.x] += v;
    }
}
}  // namespace

namespace rverom {
int adjoint_partials_capacity(rverom_t h) { return h->n_sm * 16; }
}

extern "C" int rve_rom_adjoint(rverom_t h, int64_t n_points, const int32_t *type, const double *Fbar,
                               const double *q, const double *gPbar, double *gFbar, double *gTheta,
                               int32_t *status, void *stream) {
    if (!h || n_points < 0 || n_points > INT32_MAX) return RVEROM_ERR_ARG;
    if (n_points == 0) return RVEROM_OK;
    if (!Fbar || !q || !gPbar || !gFbar || !gTheta || !status) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int cap = adjoint_partials_capacity(h);
    if (!h->partials) {
        if (cudaMalloc(&h->partials, (size_t)cap * 4 * sizeof(double)) != cudaSuccess) return RVEROM_ERR_CUDA;
        h->partials_cap = cap;
    }
    int rc = prepare_buckets(h, n_points, type, status, nullptr, st);
    if (rc != RVEROM_OK) return rc;
    for (int t = 0; t < h->n_types; ++t) {
        if (!type && t > 0) break;
        EvalArgs a = {};
        a.t = h->types[t];
        a.n_points = n_points;
        a.nmax = h->nmax;
        a.V0 = h->V0;
        a.Fbar = Fbar;
        a.q = const_cast<double *>(q);
        a.status = status;
        a.gP = gPbar;
        a.gF = gFbar;
        a.partials = h->partials;
        if (type) {
            a.perm = h->perm;
            a.count = h->bucket_small + t;
            a.offset = h->bucket_small + (RVEROM_MAX_TYPES + 1) + t;
        }
        int grid = 0;
        cudaError_t e = dispatch_adjoint(h->dim, a.t.n, a, h->n_sm, n_points, st, &grid);
        if (e != cudaSuccess || grid > h->partials_cap) return RVEROM_ERR_CUDA;
        k_theta_reduce<<<1, 32, 0, st>>>(h->partials, grid, gTheta + 4 * t);
        if (cudaGetLastError() != cudaSuccess) return RVEROM_ERR_CUDA;
    }
    return RVEROM_OK;
}
