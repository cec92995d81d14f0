// registry.h -- per-spline launch table shared by the ABI (interp.cu) and the per-spline
// instantiation units (ops_inst.cu, compiled once per spline and kernel family).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace ibr {

// launch options a handle passes to the launchers (set per handle, see interp_set_option)
enum LaunchFlags : int {
    FLAG_BIN_SMALL = 1,     // piece-binned kernels: 256-query tiles on 128-thread CTAs
    FLAG_DENSE_ON = 2,      // dense piece tables where emitted (binned evaluation and rays)
    FLAG_DENSE_OFF = 4,     // unrolled per-piece code even for the rays of dense-table splines
    FLAG_BINNED_ON = 8,     // rays: the piece-binned kernel for any multi-piece spline
    FLAG_BINNED_OFF = 16,   // rays: the plain kernel
};

using EvalFn = cudaError_t (*)(const float *, int64_t, const void *, const ibl::Layout &, float *, float *,
                               const float *, int, cudaStream_t);
using AdjFn = cudaError_t (*)(const float *, int64_t, const float *, const ibl::Layout &, float *, cudaStream_t);
using RayFn = cudaError_t (*)(const ibl::RayGeom &, const void *, const ibl::Layout &, float *, float *, int,
                              cudaStream_t);
using SortFn = cudaError_t (*)(const float *, int64_t, const ibl::Layout &, int, int, unsigned *, int, int32_t *,
                               float *, cudaStream_t);
using DbgFn = cudaError_t (*)(const float *, int64_t, const ibl::Layout &, int32_t *, int32_t *, cudaStream_t);
// the adjoint on spatially binned queries: the queries as 16-byte records (x, y, z, gout) in
// the caller's order, the query indices in bin order, bin starts, work item starts, bins per
// axis and chunk, work items at most
struct BoxArgs {
    const float *rec;
    const int *idx;
    const int *bin_start;
    const int *item_start;
    int nbins, nb[3], chunk, max_items;
    int lb;          // log2 cells per bin and axis (SplineOps::box_lb)
};
using BoxAdjFn = cudaError_t (*)(const BoxArgs &, const ibl::Layout &, float *, cudaStream_t);

struct SplineOps {
    const char *name = nullptr;
    int s = 0, nxi = 0, M = 0, D = 0, detl = 0, halo = 0, K = 0, deg = 0, nmon = 0;
    int kind = 0;                // 0: box spline M_xi; n >= 1: Voronoi spline V_n (xi = 2 G)
    const int *xi = nullptr;     // s x nxi row-major
    const int *cosets = nullptr; // M x s
    double fma_value = 0, fma_grad = 0, lookups = 0;
    int nnz_sum = 0;             // nonzeros of A_j summed over the pieces (a coset's divergent
                                 // work in a warp that meets every piece)
    bool binned_eval = false;    // evaluation defaults to the piece-binned kernels
    bool coop_eval = false;      // evaluation runs the warp-cooperative gathers
    EvalFn eval[3][3] = {};      // [storage: f32, f16, bf16][mode: value, value+grad, pullback]
    EvalFn eval_binned[3][3] = {};  // the same, piece-binned (multi-piece splines only)
    AdjFn adjoint = nullptr;
    BoxAdjFn adjoint_box = nullptr;  // 3-D splines with fewer than 4 pieces
    int box_lb = 0;                  // log2 cells per bin and axis of adjoint_box
    RayFn rays[2] = {};          // [value, value+grad], 3-D splines, FP32 storage
    DbgFn debug = nullptr;
    SortFn sort = nullptr;
};

// kernel families, one translation unit each
enum Part { PART_VALUE = 0, PART_GRAD = 1, PART_PULL = 2, PART_MISC = 3 };

}  // namespace ibr

#define INTERP_FILL_DECL(name)                     \
    namespace ibr {                                \
    void fill_##name##_0(SplineOps &);             \
    void fill_##name##_1(SplineOps &);             \
    void fill_##name##_2(SplineOps &);             \
    void fill_##name##_3(SplineOps &);             \
    }

namespace ibr {
int batch_kind_3d(const char *name);
cudaError_t batch_grid_3d(int *grid);
cudaError_t batch_launch_3d(const ibl::BatchVol *vols, int nvol, int64_t total_tiles, unsigned long long *counter,
                            int grid, cudaStream_t st);
}  // namespace ibr
