// layout.h -- device memory layout of the coefficient arrays (shared by host and device code).
//
// The coset arrays are padded by 2*HALO zero sites per side and stored together in 32-byte
// bricks.  A brick holds, for every coset k (when the coset count M is a power of two and fits),
// the same small box of 2^lb_0 x ... x 2^lb_{s-1} sites, coset-major inside the brick:
//     FP32:  M = 1: 2x2x2    M = 2 (BCC): 2x2x1 x 2 cosets    M = 4 (FCC): 2x1x1 x 4 cosets
//            4-D M = 2 (D4*): 2x2x1x1 x 2 cosets
//     16-bit: one more bit per brick (2x2x4, 2x2x2 x 2, 2x2x1 x 4, ...)
// A query's stencils on all cosets lie in the same small world-space region, so with the cosets
// side by side they share sectors; a random query then touches fewer distinct 32-byte sectors,
// and the L1 -> L2 miss requests (one per sector) are what bound the gather.
// The layout is separable:
//     offset(k, i) = k * kw + sum_a (i_a >> lb_a) * bstride_a + (i_a & (2^lb_a - 1)) * wt_a
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
    int kw;            // element offset between cosets (inside a brick, or whole arrays)
    int total;         // elements over all cosets
};

constexpr int ilog2(int v)
{
    int r = 0;
    while ((1 << (r + 1)) <= v) ++r;
    return r;
}

// can the M cosets share bricks (M a power of two, M elements fit in 32 bytes)?
constexpr bool can_interleave(int esz, int M) { return (M & (M - 1)) == 0 && M > 1 && M * esz <= 16; }

// brick width (log2) of axis a for s axes and esz-byte elements (32-byte bricks), with the M
// cosets side by side in each brick (inter) or in separate arrays: the brick's address bits,
// minus those taken by the cosets, dealt one per axis from axis 0
constexpr int brick_lb(int s, int esz, int M, bool inter, int a)
{
    int bits = ilog2(32 / esz) - (inter ? ilog2(M) : 0);
    int lb = 0;
    for (int i = 0; bits > 0; i = (i + 1) % s, --bits)
        if (i == a) ++lb;
    return lb;
}

// fill the layout for dims n (s axes), padding pad, element size esz and M cosets, interleaving
// the cosets inside the bricks if asked and possible; returns false if the padded arrays would
// not be addressable with 32-bit element offsets
inline bool make_layout(Layout &L, int s, const int *n, int pad, int esz, int M, bool interleave)
{
    const bool inter = interleave && can_interleave(esz, M);
    L.s = s;
    L.pad = pad;
    long long brick = 1;
    for (int a = 0; a < 4; ++a) {
        L.n[a] = a < s ? n[a] : 1;
        L.lb[a] = a < s ? brick_lb(s, esz, M, inter, a) : 0;
        const int w = 1 << L.lb[a];
        L.pdims[a] = a < s ? ((n[a] + 2 * pad + w - 1) / w) * w : 1;
        brick *= w;
    }
    long long wt = 1;
    for (int a = s - 1; a >= 0; --a) {
        L.wt[a] = (int)wt;
        wt *= (1 << L.lb[a]);
    }
    long long bs = inter ? brick * M : brick;
    for (int a = 3; a >= 0; --a) {
        L.bstride[a] = a < s ? (int)bs : 0;
        if (a < s) bs *= (L.pdims[a] >> L.lb[a]);
    }
    // bs is now the elements of all bricks (all cosets if interleaved, one coset otherwise)
    const long long total = inter ? bs : bs * M;
    if (total >= 0x7fffffffLL) return false;
    L.kw = inter ? (int)brick : (int)bs;
    L.total = (int)total;
    return true;
}

// one volume of a batched evaluation (device-side descriptor)
struct BatchVol {
    const float *c;          // FP32 padded, bricked coefficients
    const float *pts;        // queries (npts x s)
    float *out;              // values (npts)
    long long npts;
    long long first_tile;    // global index of the volume's first tile (prefix over volumes)
    int kind;                // index of the volume's spline in its batched kernel's spline list
    int tile;                // queries per tile (chosen per spline by the autotuner)
    Layout L;
};

// geometry of a set of orthographic rays (see interp_eval_rays)
struct RayGeom {
    float origin[3], du[3], dv[3], dir[3], lo[3], hi[3];
    int width, height, steps;
};

#if defined(__CUDACC__)
#define IBL_HD __host__ __device__ __forceinline__
#else
#define IBL_HD inline
#endif

// element offset of padded index p (s axes) of coset k
IBL_HD int elem_offset(const Layout &L, int k, const int *p)
{
    int off = k * L.kw;
    for (int a = 0; a < L.s; ++a) off += (p[a] >> L.lb[a]) * L.bstride[a] + (p[a] & ((1 << L.lb[a]) - 1)) * L.wt[a];
    return off;
}

}  // namespace ibl
