// layout.h -- device memory layout of the coefficient arrays (shared by host and device code).
//
// Each coset array is padded by 2*HALO sites per side (zeros) and stored in 32-byte bricks:
// 2x2x2 FP32 or 2x2x4 FP16/BF16 sites in 3-D, 2x2x2x1 FP32 / 2x2x2x2 16-bit in 4-D.  A random
// query's stencil then touches fewer distinct 32-byte sectors than in row-major order, and the
// L1 -> L2 miss requests (one per sector) are what bound the gather.  The layout is separable:
//     offset(i) = sum_a (i_a >> lb_a) * bstride_a + (i_a & (2^lb_a - 1)) * wt_a
// so a site's address is a sum of per-axis terms.
#pragma once

namespace ibl {

struct Layout {
    int s;
    int n[4];          // samples per axis of every coset (unpadded)
    int pad;           // padding per side (sites), 2 * HALO
    int pdims[4];      // padded samples per axis (multiple of the brick width)
    int lb[4];         // log2 of the brick width per axis
    int wt[4];         // weight of the within-brick coordinate per axis
    int bstride[4];    // elements between neighbouring bricks along each axis
    int coset_elems;   // elements of one padded coset array
};

// brick width (log2) of axis a for an s-dimensional array of esz-byte elements (32-byte bricks)
constexpr int brick_lb(int s, int esz, int a)
{
    if (s == 3) return (esz == 4) ? 1 : (a == 2 ? 2 : 1);
    if (s == 4) return (esz == 4) ? (a == 3 ? 0 : 1) : 1;
    return 0;
}

// fill the layout for dims n (s axes), padding pad and element size esz; returns false if the
// padded arrays would not be addressable with 32-bit element offsets
inline bool make_layout(Layout &L, int s, const int *n, int pad, int esz, int n_cosets)
{
    L.s = s;
    L.pad = pad;
    long long brick = 1;
    for (int a = 0; a < 4; ++a) {
        L.n[a] = a < s ? n[a] : 1;
        L.lb[a] = a < s ? brick_lb(s, esz, a) : 0;
        const int w = 1 << L.lb[a];
        L.pdims[a] = a < s ? ((n[a] + 2 * pad + w - 1) / w) * w : 1;
        brick *= w;
    }
    long long wt = 1;
    for (int a = s - 1; a >= 0; --a) {
        L.wt[a] = (int)wt;
        wt *= (1 << L.lb[a]);
    }
    long long bs = brick;
    for (int a = 3; a >= 0; --a) {
        L.bstride[a] = a < s ? (int)bs : 0;
        if (a < s) bs *= (L.pdims[a] >> L.lb[a]);
    }
    const long long total = bs * n_cosets;
    if (total >= 0x7fffffffLL) return false;
    L.coset_elems = (int)bs;
    return true;
}

#if defined(__CUDACC__)
#define IBL_HD __host__ __device__ __forceinline__
#else
#define IBL_HD inline
#endif

// element offset of padded index p (s axes) inside coset k
IBL_HD int elem_offset(const Layout &L, int k, const int *p)
{
    int off = k * L.coset_elems;
    for (int a = 0; a < L.s; ++a) off += (p[a] >> L.lb[a]) * L.bstride[a] + (p[a] & ((1 << L.lb[a]) - 1)) * L.wt[a];
    return off;
}

}  // namespace ibl
