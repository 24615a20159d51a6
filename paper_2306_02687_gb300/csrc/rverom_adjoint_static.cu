// rverom_adjoint_static.cu -- rve_rom_adjoint_static: the implicit adjoint
// (same kernel and results as rve_rom_adjoint) without any device
// allocation in the call.
//
// Why: rve_rom_adjoint keeps its per-CTA partial sums (and, for mixed-type
// batches, its per-type point lists) in workspaces that it allocates with
// cudaMalloc on first use or when a batch grows.  Some callers cannot allow
// that: a macro FE code that calls the adjoint from its per-increment
// material/element callbacks, where a cudaMalloc/cudaFree may synchronize the
// device and stall the host element loop, or a process whose device memory is
// entirely reserved by another allocator (a framework's caching allocator,
// a fixed memory pool).  This entry point uses instead a file-scope static
// device array, which every GPU that loads the library holds until the
// process exits.
//
// Scratch layout (RVEROM_STATIC_SCRATCH_BYTES in total, 256-byte aligned
// regions): per-CTA partial sums [RVEROM_STATIC_MAX_CTAS][4] double, the
// bucketing counters (3 x (RVEROM_MAX_TYPES + 1) int32) and the per-type
// point lists [RVEROM_STATIC_MAX_TYPED_POINTS] int32.
//
// Set-up: the first call on a device looks up the device address of the
// array with cudaGetSymbolAddress, with that device current, and caches it
// per device; that first call should therefore come before any stream
// capture.  All calls share the array: the counters are cleared at the start
// of every call and the partials are fully rewritten by every call, but two
// calls whose GPU work overlaps (different streams, or different threads on
// the same device) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rverom.h"
#include "rom_core.cuh"
#include "rverom_internal.h"

using namespace rverom;

namespace {

constexpr size_t kPartialsBytes = (size_t)RVEROM_STATIC_MAX_CTAS * 4 * sizeof(double);
constexpr size_t kCountersOff = kPartialsBytes;
constexpr size_t kCountersBytes = 256;  // 3 x (RVEROM_MAX_TYPES + 1) int32 fit in 256 bytes
constexpr size_t kPermOff = kCountersOff + kCountersBytes;
constexpr size_t kScratchBytes = kPermOff + (size_t)RVEROM_STATIC_MAX_TYPED_POINTS * sizeof(int32_t);
static_assert(3 * (RVEROM_MAX_TYPES + 1) * sizeof(int32_t) <= kCountersBytes, "counter region too small");
static_assert(kScratchBytes == RVEROM_STATIC_SCRATCH_BYTES, "header size out of date");

static __device__ __align__(256) unsigned char g_adjoint_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device (looked up
// once per device).
int scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return RVEROM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_adjoint_scratch) != cudaSuccess || !p) return RVEROM_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return RVEROM_OK;
}

__global__ void k_count(const int32_t *type, int64_t n, int n_types, int32_t *counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int t = type[i];
        if (t < 0 || t >= n_types) t = n_types;
        atomicAdd(&counts[t], 1);
    }
}

__global__ void k_offsets(int n_types, const int32_t *counts, int32_t *offsets, int32_t *cursor) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t o = 0;
        for (int t = 0; t <= n_types; ++t) {
            offsets[t] = o;
            cursor[t] = o;
            o += counts[t];
        }
    }
}

__global__ void k_scatter(const int32_t *type, int64_t n, int n_types, int32_t *cursor, int32_t *perm,
                          int32_t *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int t = type[i];
        if (t < 0 || t >= n_types) {
            status[i] = ST_NONFINITE;
            t = n_types;
        }
        perm[atomicAdd(&cursor[t], 1)] = (int32_t)i;
    }
}

__global__ void k_reduce(const double *partials, int nblocks, double *gTheta) {
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partials[(int64_t)b * 4 + threadIdx.x];
        gTheta[threadIdx.x] += v;
    }
}

}  // namespace

extern "C" int rve_rom_adjoint_static(rverom_t h, int64_t n_points, const int32_t *type, const double *Fbar,
                                      const double *q, const double *gPbar, double *gFbar, double *gTheta,
                                      int32_t *status, void *stream) {
    if (!h || n_points < 0 || n_points > INT32_MAX) return RVEROM_ERR_ARG;
    if (n_points == 0) return RVEROM_OK;
    if (!Fbar || !q || !gPbar || !gFbar || !gTheta || !status) return RVEROM_ERR_ARG;
    if (type && n_points > RVEROM_STATIC_MAX_TYPED_POINTS) return RVEROM_ERR_SCRATCH_LIMIT;
    // every CTA of the adjoint kernels has at least 128 threads, so at most
    // 16 are resident per SM and the persistent grid is <= 16 x SMs
    if ((int64_t)h->n_sm * 16 > RVEROM_STATIC_MAX_CTAS) return RVEROM_ERR_SCRATCH_LIMIT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RVEROM_ERR_CUDA;
    if (dev != h->device) return RVEROM_ERR_ARG;
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc != RVEROM_OK) return rc;
    double *partials = reinterpret_cast<double *>(base);
    int32_t *counts = reinterpret_cast<int32_t *>(base + kCountersOff);
    int32_t *offsets = counts + (RVEROM_MAX_TYPES + 1);
    int32_t *cursor = offsets + (RVEROM_MAX_TYPES + 1);
    int32_t *perm = reinterpret_cast<int32_t *>(base + kPermOff);
    cudaStream_t st = (cudaStream_t)stream;
    if (type) {
        if (cudaMemsetAsync(counts, 0, (RVEROM_MAX_TYPES + 1) * sizeof(int32_t), st) != cudaSuccess)
            return RVEROM_ERR_CUDA;
        int grid = (int)((n_points + 255) / 256);
        if (grid > 4 * h->n_sm) grid = 4 * h->n_sm;
        k_count<<<grid, 256, 0, st>>>(type, n_points, h->n_types, counts);
        k_offsets<<<1, 32, 0, st>>>(h->n_types, counts, offsets, cursor);
        k_scatter<<<grid, 256, 0, st>>>(type, n_points, h->n_types, cursor, perm, status);
        if (cudaGetLastError() != cudaSuccess) return RVEROM_ERR_CUDA;
    }
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
        a.partials = partials;
        if (type) {
            a.perm = perm;
            a.count = counts + t;
            a.offset = offsets + t;
        }
        int grid = 0;
        cudaError_t e = dispatch_adjoint(h->dim, a.t.n, a, h->n_sm, n_points, st, &grid);
        if (e != cudaSuccess || grid > RVEROM_STATIC_MAX_CTAS) return RVEROM_ERR_CUDA;
        k_reduce<<<1, 32, 0, st>>>(partials, grid, gTheta + 4 * t);
        if (cudaGetLastError() != cudaSuccess) return RVEROM_ERR_CUDA;
    }
    return RVEROM_OK;
}
