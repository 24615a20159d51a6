// rverom_diag.cu -- diagnostics of the library's own arithmetic and of the
// machine it runs on (no counterpart in the paper):
//   rverom_df_log      the double-float logarithm of the mixed form's micro
//                      law, evaluated at caller-given points
//   rverom_peak_probe  measured throughput of the execution units the hot
//                      path uses (FP32 FMA, FP64 FMA, tcgen05 TF32 and BF16
//                      MMAs), the denominators of the roofline fractions
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rverom.h"
#include "df64.cuh"
#include "tc.cuh"

namespace rverom {
namespace {

__global__ void k_df_log(int64_t n, const double *x, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const df v = df_from(x[i]);
        out[i] = df_to(df_log(v));
    }
}

// FMA throughput: NCH independent chains per thread, each a long sequence of
// dependent FMAs whose operands the compiler cannot fold (seed from the
// thread index, multiplier and addend from kernel arguments).
template <typename T, int NCH>
__global__ void __launch_bounds__(256) k_fma(int iters, T a, T b, T *sink) {
    T v[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < NCH; ++c) v[c] = fma(v[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += v[c];
    if (s == (T)12345.678) sink[threadIdx.x] = s;  // never true for the arguments used; keeps the chains live
}

// tcgen05 MMA throughput: one thread per CTA issues `iters` MMAs of
// M = 128, N = 256 (K = 8 TF32 or 16 BF16 values, 32 bytes per row) from
// zero-filled shared-memory operands into a 256-column TMEM accumulator,
// commits them to an mbarrier and waits (bounded) for their completion.
template <bool BF16>
__global__ void __launch_bounds__(128, 1) k_mma(int iters, int *err) {
    __shared__ __align__(1024) float sA[128 * 8];
    __shared__ __align__(1024) float sB[256 * 8];
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < 128 * 8; i += blockDim.x) sA[i] = 0.0f;
    for (int i = tid; i < 256 * 8; i += blockDim.x) sB[i] = 0.0f;
    if (warp == 0) {
        tc::tmem_alloc(&slot, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_init_fence();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = slot;
    if (tid == 0) {
        // operand layout: [k group of 16 bytes][row group of 8][8 rows][16 bytes]
        const uint64_t ad = tc::smem_desc(tc::smem_u32(sA), 128 * 16, 128);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sB), 256 * 16, 128);
        const uint32_t id = BF16 ? ((1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24))
                                 : tc::idesc_tf32(128, 256);
        for (int it = 0; it < iters; ++it) {
            if (BF16) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(id), "r"(it > 0 ? 1u : 0u)
                    : "memory");
            } else {
                tc::mma_tf32(tmem, ad, bd, id, it > 0 ? 1u : 0u);
            }
        }
        tc::mma_commit(&bar);
        if (!tc::mbar_wait(&bar, 0)) atomicExch(err, 1);
    }
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 256);
    }
}

}  // namespace
}  // namespace rverom

using namespace rverom;

extern "C" int rverom_df_log(int64_t n, const double *x, double *out, void *stream) {
    if (n < 0 || (n > 0 && (!x || !out))) return RVEROM_ERR_ARG;
    if (n == 0) return RVEROM_OK;
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_df_log<<<grid, 256, 0, (cudaStream_t)stream>>>(n, x, out);
    return cudaGetLastError() == cudaSuccess ? RVEROM_OK : RVEROM_ERR_CUDA;
}

extern "C" int rverom_peak_probe(int32_t unit, double *tflops, void *stream) {
    if (!tflops || unit < 0 || unit > 3) return RVEROM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RVEROM_ERR_CUDA;
    void *scratch = nullptr;
    if (cudaMalloc(&scratch, 4096) != cudaSuccess) return RVEROM_ERR_CUDA;
    int *err = reinterpret_cast<int *>(scratch);
    cudaMemsetAsync(scratch, 0, 4096, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    int rc = RVEROM_OK;
    for (int rep = 0; rep < 4 && rc == RVEROM_OK; ++rep) {
        double flop = 0.0;
        cudaEventRecord(e0, st);
        if (unit == 0) {
            const int iters = 4096, blocks = n_sm * 8;
            k_fma<float, 8><<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f, reinterpret_cast<float *>(scratch) + 64);
            flop = 2.0 * blocks * 256.0 * iters * 16.0 * 8.0;
        } else if (unit == 1) {
            const int iters = 256, blocks = n_sm * 8;
            k_fma<double, 8><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, reinterpret_cast<double *>(scratch) + 64);
            flop = 2.0 * blocks * 256.0 * iters * 16.0 * 8.0;
        } else {
            const int iters = 8192, blocks = n_sm;
            if (unit == 2) k_mma<false><<<blocks, 128, 0, st>>>(iters, err);
            else k_mma<true><<<blocks, 128, 0, st>>>(iters, err);
            flop = 2.0 * blocks * (double)iters * 128.0 * 256.0 * (unit == 2 ? 8.0 : 16.0);
        }
        cudaEventRecord(e1, st);
        float ms = 0.0f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = RVEROM_ERR_CUDA;
            break;
        }
        if (rep > 0 && ms > 0.0f && flop / (ms * 1e-3) / 1e12 > best) best = flop / (ms * 1e-3) / 1e12;
    }
    int h_err = 0;
    if (rc == RVEROM_OK && cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = RVEROM_ERR_CUDA;
    if (rc == RVEROM_OK && h_err) rc = RVEROM_ERR_CUDA;  // an MMA wait timed out
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    *tflops = rc == RVEROM_OK ? best : 0.0;
    return rc;
}
