// rverom_internal.h -- handle layouts shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rverom.h"
#include "rom_core.cuh"
#include "rom_ws.cuh"
#include "rom_tc.cuh"
#include "rom_tc_ws.cuh"
#include "rom_tc_wide.cuh"

struct rverom_s {
    int dim = 2;
    int n_types = 0;
    int nmax = 0;
    int n_sm = 1;
    int device = 0;
    double V0 = 1.0;
    rverom::TypeDev types[RVEROM_MAX_TYPES] = {};
    int32_t *bucket_small = nullptr;  // counts | offsets | cursor, each n_types+1
    int32_t *perm = nullptr;          // point lists of a mixed batch
    int64_t perm_cap = 0;
    double *partials = nullptr;       // per-CTA partial sums of the adjoint
    int64_t partials_cap = 0;
    int choice[RVEROM_MAX_TYPES][2] = {};  // forward kernel candidate per type and precision
    float *cond = nullptr;            // per-point workspace records of the tensor-core form
    int64_t cond_cap = 0;             // in floats
    int cond_words = 0;               // record size (floats) of the largest tensor-core configuration
};

namespace rverom {

// Launch one compiled tile configurations <D, NA, TA, TB, NP, CI, KT> as a
// persistent grid of at most (SMs x resident CTAs) blocks.
template <int D, int NA, int TA, int TB, int NP, int CI, typename KT, bool ADJ, bool SYM = false>
cudaError_t launch_cfg(const EvalArgs &a, int n_sm, int64_t max_points, cudaStream_t st, int *grid_out) {
    using PL = Plan<D, NA, TA, TB, NP, CI, KT, SYM>;
    auto kern = eval_kernel<D, NA, TA, TB, NP, CI, KT, ADJ, SYM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PL::NT, PL::bytes);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t tiles = (max_points + NP - 1) / NP;
    int64_t grid = (int64_t)n_sm * occ;
    if (tiles < grid) grid = tiles;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, PL::NT, PL::bytes, st>>>(a);
    return cudaGetLastError();
}

// Warp-specialized mixed-precision forward kernel <D, NA, TA, TB, NP, CI>.
template <int D, int NA, int TA, int TB, int NP, int CI>
cudaError_t launch_ws(const EvalArgs &a, int n_sm, int64_t max_points, cudaStream_t st, int *grid_out) {
    using PL = WsPlan<D, NA, TA, TB, NP, CI>;
    auto kern = eval_ws_kernel<D, NA, TA, TB, NP, CI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PL::NT, PL::bytes);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t tiles = (max_points + NP - 1) / NP;
    int64_t grid = (int64_t)n_sm * occ;
    if (tiles < grid) grid = tiles;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, PL::NT, PL::bytes, st>>>(a);
    return cudaGetLastError();
}

// Tensor-core mixed-precision forward kernel <D, NA, NP, CI> (one CTA per
// SM: its shared memory and TMEM allocation fill the SM), followed by the
// per-thread condensation of its workspace records.
template <int D, int NA, int NP, int CI>
cudaError_t launch_tc(const EvalArgs &a, int n_sm, int64_t max_points, cudaStream_t st, int *grid_out) {
    using PL = TcPlan<D, NA, NP, CI>;
    constexpr int CT = 32, TPP = 8;
    using CP = CondPlan<D, NA, CT, TPP>;
    if (!a.t.Bimg || a.t.img_nn != PL::NN || !a.cond) return cudaErrorInvalidValue;
    auto kern = eval_tc_kernel<D, NA, NP, CI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes);
    if (e != cudaSuccess) return e;
    auto ckern = condense_kernel<D, NA, CT, TPP>;
    e = cudaFuncSetAttribute(ckern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CP::bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ckern, CT * TPP, CP::bytes);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t tiles = (max_points + NP - 1) / NP;
    int64_t grid = n_sm;
    if (tiles < grid) grid = tiles;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, PL::NT, PL::bytes, st>>>(a);
    int64_t cgrid = (max_points + CT - 1) / CT, cmax = (int64_t)n_sm * occ;
    if (cgrid > cmax) cgrid = cmax;
    if (cgrid < 1) cgrid = 1;
    ckern<<<(unsigned)cgrid, CT * TPP, CP::bytes, st>>>(a);
    return cudaGetLastError();
}
// warp-specialized tensor-core kernel (8 tile warps, 4 helper warps) and the
// same condensation kernel; refuses to launch if the compiled register count
// differs from the allocation its in-kernel register split assumes
template <int D, int NA, int NP, int CI>
cudaError_t launch_tc_ws(const EvalArgs &a, int n_sm, int64_t max_points, cudaStream_t st, int *grid_out) {
    using PL = TcWsPlan<D, NA, NP, CI>;
    constexpr int CT = 32, TPP = 8;
    using CP = CondPlan<D, NA, CT, TPP>;
    if (!a.t.Bimg || a.t.img_nn != PL::NN || !a.cond) return cudaErrorInvalidValue;
    auto kern = eval_tc_ws_kernel<D, NA, NP, CI>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != PL::REGS_LAUNCH) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes);
    if (e != cudaSuccess) return e;
    auto ckern = condense_kernel<D, NA, CT, TPP>;
    e = cudaFuncSetAttribute(ckern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CP::bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ckern, CT * TPP, CP::bytes);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t tiles = (max_points + NP - 1) / NP;
    int64_t grid = n_sm;
    if (tiles < grid) grid = tiles;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, PL::NT, PL::bytes, st>>>(a);
    int64_t cgrid = (max_points + CT - 1) / CT, cmax = (int64_t)n_sm * occ;
    if (cgrid > cmax) cgrid = cmax;
    if (cgrid < 1) cgrid = 1;
    ckern<<<(unsigned)cgrid, CT * TPP, CP::bytes, st>>>(a);
    return cudaGetLastError();
}
// tensor-core kernel for wide planar ROMs (NA = 36 or 68) and the
// condensation kernel (CT points per CTA, so that its shared-memory copy of
// the augmented systems fits)
template <int D, int NA, int CI, int FK>
cudaError_t launch_tc_wide(const EvalArgs &a, int n_sm, int64_t max_points, cudaStream_t st, int *grid_out) {
    using PL = TcWidePlan<D, NA, CI, FK>;
    constexpr int CT = NA <= 36 ? 32 : 8, TPP = 256 / CT;
    using CP = CondPlan<D, NA, CT, TPP>;
    static_assert(CP::bytes <= 227 * 1024, "condensation shared memory");
    if (!a.t.Bimg || a.t.img_nn != PL::NN || !a.cond) return cudaErrorInvalidValue;
    auto kern = eval_tc_wide_kernel<D, NA, CI, FK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes);
    if (e != cudaSuccess) return e;
    auto ckern = condense_kernel<D, NA, CT, TPP>;
    e = cudaFuncSetAttribute(ckern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CP::bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ckern, CT * TPP, CP::bytes);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int64_t tiles = (max_points + PL::NP - 1) / PL::NP;
    int64_t grid = n_sm;
    if (tiles < grid) grid = tiles;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, PL::NT, PL::bytes, st>>>(a);
    int64_t cgrid = (max_points + CT - 1) / CT, cmax = (int64_t)n_sm * occ;
    if (cgrid > cmax) cgrid = cmax;
    if (cgrid < 1) cgrid = 1;
    ckern<<<(unsigned)cgrid, CT * TPP, CP::bytes, st>>>(a);
    return cudaGetLastError();
}
int tc_record_words(int dim, int n);
int tc_image_nn(int dim, int n);

// Tile configuration of the adjoint (float64 form) per (dimension, n~ bucket).
inline cudaError_t dispatch_adjoint(int dim, int n, const EvalArgs &a, int n_sm, int64_t max_points,
                                    cudaStream_t st, int *grid_out) {
    if (dim == 2) {
        if (n <= 12) return launch_cfg<2, 16, 4, 4, 16, 8, double, true>(a, n_sm, max_points, st, grid_out);
        if (n <= 16) return launch_cfg<2, 20, 5, 5, 16, 8, double, true>(a, n_sm, max_points, st, grid_out);
        if (n <= 24) return launch_cfg<2, 28, 7, 7, 8, 8, double, true>(a, n_sm, max_points, st, grid_out);
        if (n <= 32) return launch_cfg<2, 36, 9, 9, 8, 8, double, true>(a, n_sm, max_points, st, grid_out);
        if (n <= 64) return launch_cfg<2, 72, 9, 9, 2, 8, double, true>(a, n_sm, max_points, st, grid_out);
    } else if (dim == 3) {
        if (n <= 47) return launch_cfg<3, 56, 7, 7, 2, 4, double, true>(a, n_sm, max_points, st, grid_out);
    }
    return cudaErrorInvalidValue;
}
bool supported_modes(int dim, int n);
int prepare_buckets(rverom_t h, int64_t n, const int32_t *type, int32_t *status, double *rnorm,
                    cudaStream_t st);

// Candidate forward kernels (tile configurations) of an RVE type; entry 0 is
// the default before autotuning.  Returns the number of candidates; `info`
// (optional) receives each candidate's name and kernel launches per type.
using LaunchFn = cudaError_t (*)(const EvalArgs &, int, int64_t, cudaStream_t, int *);
struct CandInfo {
    const char *name;
    int launches;
};
int forward_candidates(int dim, int n, bool mixed, LaunchFn *out, int max_out, CandInfo *info = nullptr);
}  // namespace rverom
