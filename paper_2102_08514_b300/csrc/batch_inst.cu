// batch_inst.cu -- the persistent batched kernel over the 3-D splines listed in
// INTERP_GEN_BATCH_3D, and the lookup of a spline name in that list.
#include "kernels.cuh"
#include "registry.h"

#define IB_LIST INTERP_GEN_BATCH_3D
#define IB_NAMES INTERP_GEN_BATCH_NAMES_3D
#define IB_FN(x) x##_3d

namespace ibr {

// spline-list index of `name` in this dimension's batched kernel, or -1
int IB_FN(batch_kind)(const char *name)
{
    static const char *const names[] = {IB_NAMES};
    for (int i = 0; i < (int)(sizeof(names) / sizeof(names[0])); ++i) {
        const char *a = names[i], *b = name;
        while (*a && *a == *b) { ++a; ++b; }
        if (*a == 0 && *b == 0) return i;
    }
    return -1;
}

// CTAs of the persistent kernel that fit on the device at once (grid size of one wave)
cudaError_t IB_FN(batch_grid)(int *grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ib::k_batch<IB_LIST>, 128, 0);
    *grid = sms * (per_sm > 0 ? per_sm : 1);
    return e;
}

cudaError_t IB_FN(batch_launch)(const ibl::BatchVol *vols, int nvol, int64_t total_tiles,
                                unsigned long long *counter, int grid, cudaStream_t st)
{
    ib::k_batch<IB_LIST><<<grid, 128, 0, st>>>(vols, nvol, total_tiles, counter);
    return cudaPeekAtLastError();
}

}  // namespace ibr
