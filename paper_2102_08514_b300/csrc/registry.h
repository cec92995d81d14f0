// registry.h -- per-spline launch table shared by the ABI (interp.cu) and the per-spline
// instantiation units (ops_inst.cu, compiled once per spline and kernel family).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace ibr {

using EvalFn = cudaError_t (*)(const float *, int64_t, const void *, const ibl::Layout &, float *, float *,
                               const float *, cudaStream_t);
using AdjFn = cudaError_t (*)(const float *, int64_t, const float *, const ibl::Layout &, float *, cudaStream_t);
using DbgFn = cudaError_t (*)(const float *, int64_t, const ibl::Layout &, int32_t *, int32_t *, cudaStream_t);

struct SplineOps {
    const char *name = nullptr;
    int s = 0, nxi = 0, M = 0, D = 0, detl = 0, halo = 0, K = 0, deg = 0, nmon = 0;
    const int *xi = nullptr;     // s x nxi row-major
    const int *cosets = nullptr; // M x s
    double fma_value = 0, fma_grad = 0, lookups = 0;
    EvalFn eval[3][3] = {};      // [storage: f32, f16, bf16][mode: value, value+grad, pullback]
    AdjFn adjoint = nullptr;
    DbgFn debug = nullptr;
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
