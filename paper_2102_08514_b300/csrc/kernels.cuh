// kernels.cuh -- sm_103a kernels of the lattice convolution-sum evaluator.
//
// One thread evaluates one query point.  Per coset k it runs the steps of Algorithm 1 (Sec. 4.3)
// with the design choices below:
//   1. shift to the region of evaluation (Sec. 4.1, rho): the nearest site i of coset k and the
//      offset y = x - l_k - D i in [-D/2, D/2)^s, computed exactly (integer floor, exact FP32
//      remainder), so the cell index is bit-exact;
//   2. symmetry fold (Sec. 4.2's reflection, taken to the full signed-permutation group): y' = |y|
//      sorted descending by a sorting network; the signed permutation S is carried as per-slot
//      signed strides, which is the renaming map pi of Sec. 4.3 applied to gather addresses;
//   3. branch-free sub-region index: q = sum_i [p_i . y' - d_i >= 0] 2^i, j = sigma[q] (Sec. 4.2;
//      the table is uncompressed, 2^Q entries: up to 64 packed into 64-bit constants, 16 four-bit
//      entries each, larger ones a byte table in device memory);
//   4. gather the piece's stencil c_m = c_k[i + S^-1 g_m] (Sec. 4.1, C_0(S_j));
//   5. b = A_j c (per-monomial coefficients; A_j's nonzeros are compile-time FMA immediates), then
//      nested Horner in t = y' - anchor_j (the greedy Horner of Sec. 4.1), optionally carrying all
//      partial derivatives, mapped back through S^T.
// Tables come from the generated header (exact rationals rounded once to FP32).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <type_traits>
#include <utility>

#include "generated/splines.h"
#include "layout.h"

namespace ib {

// ------------------------------------------------------------------------------------ helpers

template <class F, int... Is>
__device__ __forceinline__ void sfor_impl(F &&f, std::integer_sequence<int, Is...>)
{
    (f(std::integral_constant<int, Is>{}), ...);
}
// calls f(integral_constant<int, I>) for I = 0 .. N-1, fully unrolled at compile time
template <int N, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    if constexpr (N > 0) sfor_impl(f, std::make_integer_sequence<int, N>{});
}

constexpr int nmon(int s, int d)
{
    long r = 1;
    for (int i = 1; i <= s; ++i) r = r * (d + i) / i;
    return (int)r;
}
// offset of block k inside the nested-Horner layout of (nv variables, degree d)
constexpr int block_off(int nv, int d, int k)
{
    int o = 0;
    for (int kk = 0; kk < k; ++kk) o += nmon(nv - 1, d - kk);
    return o;
}

template <class CT> __device__ __forceinline__ float load_coef(const CT *p)
{
    if constexpr (std::is_same_v<CT, float>) return __ldg(p);
    else if constexpr (std::is_same_v<CT, __half>) return __half2float(__ldg(p));
    else return __bfloat162float(__ldg(p));
}

// ------------------------------------------------------------------------------------ polynomial kernels

// value of the polynomial with coefficients b[OFF ..] in variables t[S-NV .. S-1] (nested Horner)
template <int S, int NV, int DEG, int OFF, int NM>
__device__ __forceinline__ float horner(const float (&b)[NM], const float (&t)[S])
{
    if constexpr (NV == 0) {
        return b[OFF];
    } else {
        constexpr int V = S - NV;
        float acc = horner<S, NV - 1, 0, OFF + block_off(NV, DEG, DEG), NM>(b, t);
        sfor<DEG>([&](auto I) {
            constexpr int k = DEG - 1 - decltype(I)::value;
            acc = fmaf(acc, t[V], horner<S, NV - 1, DEG - k, OFF + block_off(NV, DEG, k), NM>(b, t));
        });
        return acc;
    }
}

template <int NV> struct VG {
    float v;
    float g[NV > 0 ? NV : 1];
};

// value and the NV partial derivatives (variables t[S-NV .. S-1]) by nested Horner
template <int S, int NV, int DEG, int OFF, int NM>
__device__ __forceinline__ VG<NV> horner_grad(const float (&b)[NM], const float (&t)[S])
{
    VG<NV> r;
    if constexpr (NV == 0) {
        r.v = b[OFF];
    } else {
        constexpr int V = S - NV;
        VG<NV - 1> top = horner_grad<S, NV - 1, 0, OFF + block_off(NV, DEG, DEG), NM>(b, t);
        r.v = top.v;
        r.g[0] = 0.0f;
        sfor<NV - 1>([&](auto I) { r.g[1 + I] = top.g[I]; });
        sfor<DEG>([&](auto I) {
            constexpr int k = DEG - 1 - decltype(I)::value;
            VG<NV - 1> p = horner_grad<S, NV - 1, DEG - k, OFF + block_off(NV, DEG, k), NM>(b, t);
            if constexpr (k == DEG - 1) r.g[0] = r.v;              // d/dt of the leading term
            else r.g[0] = fmaf(r.g[0], t[V], r.v);
            r.v = fmaf(r.v, t[V], p.v);
            sfor<NV - 1>([&](auto J) { r.g[1 + J] = fmaf(r.g[1 + J], t[V], p.g[J]); });
        });
    }
    return r;
}

// all monomials of degree <= DEG in t[S-NV ..], scaled by `scale`, in the nested-Horner layout
template <int S, int NV, int DEG, int OFF, int NM>
__device__ __forceinline__ void monomials(float (&mu)[NM], const float (&t)[S], float scale)
{
    if constexpr (NV == 0) {
        mu[OFF] = scale;
    } else {
        constexpr int V = S - NV;
        float p = scale;
        sfor<DEG + 1>([&](auto I) {
            constexpr int k = decltype(I)::value;
            monomials<S, NV - 1, DEG - k, OFF + block_off(NV, DEG, k), NM>(mu, t, p);
            if constexpr (k < DEG) p *= t[V];
        });
    }
}

// b[MON] (+)= c[SITE] * VAL for every nonzero of a piece (pack expansion, no table indexing)
template <int NS, int NM, int SITE, int MON, float VAL, int FIRST, int SF, int SL>
__device__ __forceinline__ void nz_accum(float (&b)[NM], const float (&c)[NS], interp_gen::nz<SITE, MON, VAL, FIRST, SF, SL>)
{
    if constexpr (FIRST) b[MON] = c[SITE] * VAL;
    else b[MON] = fmaf(c[SITE], VAL, b[MON]);
}
template <int NS, int NM, class... Z>
__device__ __forceinline__ void accumulate(float (&b)[NM], const float (&c)[NS], interp_gen::nzlist<Z...>)
{
    (nz_accum<NS, NM>(b, c, Z{}), ...);
}

// ------------------------------------------------------------------------------------ geometry

// exact shift to the region of evaluation along one axis: i = floor((x - l)/D + 1/2),
// y = x - l - D i in [-D/2, D/2)
template <int D, int L>
__device__ __forceinline__ void reduce_axis(float x, int &i, float &y)
{
    const float fl = floorf(x);
    const float fr = x - fl;                 // exact, in [0, 1)
    const int v = __float2int_rz(fl) - L;    // saturates for huge |x|: then out of range
    int w;
    if constexpr (D % 2 == 0) w = v + D / 2;
    else w = v + (D - 1) / 2 + (fr >= 0.5f ? 1 : 0);
    if constexpr (D == 1) i = w;
    else if constexpr (D == 2) i = w >> 1;   // arithmetic shift = floor division
    else i = (w >= 0) ? w / D : -((-w + D - 1) / D);
    y = (float)(v - D * i) + fr;
}

// same with a run-time coset shift l
template <int D>
__device__ __forceinline__ void reduce_axis_rt(float x, int l, int &i, float &y)
{
    const float fl = floorf(x);
    const float fr = x - fl;
    const int v = __float2int_rz(fl) - l;
    int w;
    if constexpr (D % 2 == 0) w = v + D / 2;
    else w = v + (D - 1) / 2 + (fr >= 0.5f ? 1 : 0);
    if constexpr (D == 1) i = w;
    else if constexpr (D == 2) i = w >> 1;
    else i = (w >= 0) ? w / D : -((-w + D - 1) / D);
    y = (float)(v - D * i) + fr;
}

// coset shifts packed into one 64-bit word (coset_bits per entry, entries lie in [0, D)), so a
// run-time coset index can read them
template <class SP>
constexpr int coset_bits()
{
    int b = 1;
    while ((1 << b) < SP::D) ++b;
    return b;
}

template <class SP>
constexpr uint64_t cosets_packed()
{
    uint64_t v = 0;
    for (int k = 0; k < SP::M; ++k)
        for (int a = 0; a < SP::S; ++a) v |= (uint64_t)SP::COSET[k][a] << (coset_bits<SP>() * (k * SP::S + a));
    return v;
}

// one slot of the folded offset: |y| and what the gather needs about the original axis it came
// from.  d[] holds, for the folded offsets o = -2, -1, +1, +2 along the slot, the element-offset
// change from the cell's own site to the site o steps away (o steps along the slot are sg * o
// steps along the original axis; in the bricked layout the change depends on the cell's
// within-brick coordinate p).  The deltas are formed once per axis before the sort and travel
// with the slot, so each stencil site's address is the fold's base plus one delta per nonzero
// offset; entries a spline never uses are dead code.
struct Slot {
    float y;
    int sg;     // +1 / -1: sign of y along the original axis
    int ax;     // original axis
    int p;      // within-brick coordinate of the cell's padded index along that axis
    int d[4];   // offset deltas of o = -2, -1, +1, +2 (index o + 2, or o + 1 for o > 0)
};

constexpr int delta_index(int o) { return o < 0 ? o + 2 : o + 1; }

// element-offset change of a step of D sites along an axis of brick width 2^LB, brick stride bs
// and within-brick weight wt, from a site whose within-brick coordinate is e (0 <= e < 2^LB)
template <int LB, int D>
__device__ __forceinline__ int brick_delta(int e, int bs, int wt)
{
    if constexpr (LB == 0) {
        return D * bs;
    } else if constexpr (LB == 1 && (D == 2 || D == -2)) {
        return D / 2 * bs;
    } else if constexpr (LB == 1 && D == 1) {
        return wt + e * (bs - 2 * wt);              // e = 0: next site in the brick; e = 1: next brick
    } else if constexpr (LB == 1 && D == -1) {
        return wt - bs + e * (bs - 2 * wt);         // e = 0: previous brick; e = 1: previous site
    } else {
        constexpr int W = 1 << LB;
        const int v = e + D;
        return (v >> LB) * bs + ((v & (W - 1)) - e) * wt;
    }
}

// the same with a run-time brick width (the binned kernels rebuild slots from packed records)
__device__ __forceinline__ int brick_delta_rt(int e, int D, int lb, int bs, int wt)
{
    const int v = e + D;
    return (v >> lb) * bs + ((v & ((1 << lb) - 1)) - e) * wt;
}

// whether any stencil site of any piece of SP lies o steps from the cell along some folded slot
template <class SP>
constexpr bool uses_offset(int o)
{
    for (int j = 0; j < SP::K; ++j)
        for (int m = 0; m < SP::NS[j]; ++m)
            for (int a = 0; a < SP::S; ++a)
                if (SP::SITE[j][m][a] == o) return true;
    return false;
}

// the deltas of slot sl for the offsets SP uses, given its sign and within-brick coordinate e
template <class SP, int LB>
__device__ __forceinline__ void slot_deltas(Slot &sl, int e, int bs, int wt)
{
    sfor<2>([&](auto I) {
        constexpr int o = decltype(I)::value + 1;   // |o| = 1, 2
        if constexpr (uses_offset<SP>(o) || uses_offset<SP>(-o)) {
            const int fwd = brick_delta<LB, o>(e, bs, wt), bwd = brick_delta<LB, -o>(e, bs, wt);
            if constexpr (uses_offset<SP>(o)) sl.d[delta_index(o)] = sl.sg > 0 ? fwd : bwd;
            if constexpr (uses_offset<SP>(-o)) sl.d[delta_index(-o)] = sl.sg > 0 ? bwd : fwd;
        }
    });
}

template <class SP>
__device__ __forceinline__ void slot_deltas_rt(Slot &sl, int lb, int bs, int wt)
{
    sfor<2>([&](auto I) {
        constexpr int o = decltype(I)::value + 1;
        if constexpr (uses_offset<SP>(o)) sl.d[delta_index(o)] = brick_delta_rt(sl.p, sl.sg * o, lb, bs, wt);
        if constexpr (uses_offset<SP>(-o)) sl.d[delta_index(-o)] = brick_delta_rt(sl.p, -sl.sg * o, lb, bs, wt);
    });
}

// Ties are decided as for the point x + eps v, eps -> 0+, with the fixed world direction
// v = (1, 2^-12, 2^-24, 2^-36) (the direction the oracle uses), so that every coset takes the same
// side of a plane through x: values are continuous there, but a C^0 spline's gradient is not, and
// cosets deciding independently would sum one-sided gradients of different sides.
// |y_a + eps v_a| = |y_a| + eps sg_a v_a: on |y_a| = |y_b| the slot with the larger sg v comes
// first; sg (4 - ax) orders sg v the same way (v decreases with the axis).
// Only a spline that is not C^1 needs the tie rule in the sort (TIE): for a C^1 spline either
// order gives the same value and gradient on a fold wall.
template <bool TIE>
__device__ __forceinline__ void cswap(Slot &a, Slot &b)
{
    // descending order of |y| (and of sg v[ax] on ties if TIE)
    bool sw = a.y < b.y;
    if constexpr (TIE) sw |= a.y == b.y && a.sg * (4 - a.ax) < b.sg * (4 - b.ax);
    const Slot lo = sw ? a : b;
    const Slot hi = sw ? b : a;
    a = hi;
    b = lo;
}

template <int S, bool TIE>
__device__ __forceinline__ void sort_desc(Slot (&sl)[S])
{
    if constexpr (S == 2) {
        cswap<TIE>(sl[0], sl[1]);
    } else if constexpr (S == 3) {
        cswap<TIE>(sl[0], sl[1]); cswap<TIE>(sl[1], sl[2]); cswap<TIE>(sl[0], sl[1]);
    } else if constexpr (S == 4) {
        cswap<TIE>(sl[0], sl[1]); cswap<TIE>(sl[2], sl[3]); cswap<TIE>(sl[0], sl[2]); cswap<TIE>(sl[1], sl[3]);
        cswap<TIE>(sl[1], sl[2]);
    }
}

// word W of sigma packed 16 four-bit entries to a 64-bit word (R <= 64, K <= 15)
template <class SP, int W>
constexpr uint64_t sigma_word()
{
    uint64_t v = 0;
    for (int r = 16 * W; r < SP::R && r < 16 * (W + 1); ++r)
        v |= (uint64_t)(SP::SIGMA[r] < 0 ? 15 : SP::SIGMA[r]) << (4 * (r - 16 * W));
    return v;
}

// ------------------------------------------------------------------------------------ volume

template <class CT> struct DevVol {
    const CT *c;        // padded, bricked coset arrays, coset-major
    ibl::Layout L;
};

template <int S> struct Fold {
    int base;           // element offset of the cell's own site (coset included)
    float t[S];         // folded offset y' (before the anchor shift)
    Slot sl[S];         // per folded slot: sign, original axis, offset deltas
    int piece;
    bool in_range;
};

// element offset, relative to Fold::base, of the site displaced by a run-time o along folded
// slot sl, whose axis has brick width 2^lb, brick stride bs and within-brick weight wt
__device__ __forceinline__ int slot_term_rt(const Slot &sl, int o, int lb, int bs, int wt)
{
    return brick_delta_rt(sl.p, sl.sg * o, lb, bs, wt);
}

// log2 brick width of axis a of the S-axis layout of SP's cosets with element type CT
template <class SP, class CT>
constexpr int axis_lb(int a)
{
    return ibl::brick_lb(SP::S, (int)sizeof(CT), SP::M, false, a);
}

// Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b) (round to nearest; the _rn intrinsics
// keep the compiler from contracting or reassociating the steps)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sign (-1, 0, +1) of the exact sum of N FP32 terms, in FP32 only: Shewchuk's grow-expansion
// keeps the running sum as an expansion of N nonoverlapping components (increasing magnitude,
// zeros allowed) whose exact sum is the exact sum of the terms; the sign of a nonoverlapping
// expansion is the sign of its largest nonzero component.  No overflow for the plane tests
// (terms of magnitude <= 5/2).
template <int N>
__device__ __forceinline__ int exact_sum_sign(const float (&t)[N])
{
    float e[N];
    e[0] = t[0];
    sfor<N - 1>([&](auto I) {
        constexpr int m = decltype(I)::value + 1;          // components so far
        float q = t[m];
        sfor<m>([&](auto J) {
            float s, h;
            two_sum(q, e[J], s, h);
            e[J] = h;
            q = s;
        });
        e[m] = q;
    });
    int sg = 0;
    sfor<N>([&](auto J) {
        if (e[J] != 0.0f) sg = e[J] > 0.0f ? 1 : -1;       // the last nonzero is the largest
    });
    return sg;
}

// side of plane I for the folded offset in the slots, exactly (FP32 error-free sums: the terms
// are +-y'_a and -e); exactly on the plane, the side of y' + eps v' with v' the folded image of
// the world direction v (the term of the smallest original axis decides, v being lexicographic)
template <class SP, int I, int S>
__device__ __forceinline__ bool plane_side_exact(const Slot (&sl)[S])
{
    float terms[S + 1];
    terms[0] = -SP::PLANE_E[I];
    int best_ax = 99, sgn = 1;
    sfor<S>([&](auto A) {
        constexpr int p = SP::PLANE_P[I][decltype(A)::value];
        static_assert(p >= -1 && p <= 1, "plane normals have entries in {-1, 0, 1}");
        terms[1 + A] = p > 0 ? sl[A].y : (p < 0 ? -sl[A].y : 0.0f);
        if constexpr (p != 0) {
            if (sl[A].ax < best_ax) {
                best_ax = sl[A].ax;
                sgn = p * sl[A].sg;
            }
        }
    });
    const int d = exact_sum_sign<S + 1>(terms);
    return d != 0 ? d > 0 : sgn > 0;
}

// steps 1-3 for coset K of spline SP (K < 0: the run-time coset index kr)
template <class SP, int K, class CT>
__device__ __forceinline__ Fold<SP::S> fold_coset(const float (&x)[SP::S], const DevVol<CT> &v, int kr = 0)
{
    constexpr int S = SP::S;
    constexpr int H = SP::HALO;
    Fold<S> f;
    bool ok = true;
    int base = (K >= 0 ? K : kr) * v.L.kw;
    sfor<S>([&](auto A) {
        constexpr int a = decltype(A)::value;
        constexpr int LB = axis_lb<SP, CT>(a);      // the layout's brick width (make_layout)
        int idx;
        float y;
        if constexpr (K >= 0) {
            reduce_axis<SP::D, SP::COSET[K][a]>(x[a], idx, y);
        } else {
            constexpr int B = coset_bits<SP>();
            static_assert(SP::M * S * B <= 64, "the coset shifts must pack into 64 bits");
            constexpr uint64_t packed = cosets_packed<SP>();
            const int l = (int)((packed >> (B * (kr * S + a))) & ((1u << B) - 1u));
            reduce_axis_rt<SP::D>(x[a], l, idx, y);
        }
        ok &= (unsigned)(idx + H) < (unsigned)(v.L.n[a] + 2 * H);
        const int P = idx + 2 * H;                       // padded index of the cell's site
        const int e = P & ((1 << LB) - 1);
        const int bs = v.L.bstride[a], wt = v.L.wt[a];
        base += (P >> LB) * bs + e * wt;
        Slot &sl = f.sl[a];
        sl.y = fabsf(y);
        sl.sg = (y < 0.0f) ? -1 : 1;
        sl.ax = a;
        sl.p = e;
        slot_deltas<SP, LB>(sl, e, bs, wt);
    });
    sort_desc<S, (SP::SMOOTH < 1)>(f.sl);
    sfor<S>([&](auto A) { f.t[A] = f.sl[A].y; });
    int j = 0;
    if constexpr (SP::K > 1) {
        unsigned q = 0;
        sfor<SP::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr float e = SP::PLANE_E[i];
            float acc = -e;
            sfor<S>([&](auto A) {
                constexpr int p = SP::PLANE_P[i][decltype(A)::value];
                if constexpr (p != 0) acc = fmaf((float)p, f.t[A], acc);
            });
            // the FP32 value is within 2^-19 of p . y' - e (|p_a| = 1, y' <= 1, |e| <= 5/2 for
            // every built-in table); near zero decide exactly
            bool ge = acc >= 0.0f;
            if (fabsf(acc) <= 0x1p-17f) ge = plane_side_exact<SP, i>(f.sl);
            q |= (ge ? 1u : 0u) << i;
        });
        if constexpr (SP::R > 64) {
            j = (int)SP::sigma_at(q);                   // byte table in device memory
        } else {
            static_assert(SP::K <= 15, "sigma packing holds four-bit piece indices");
            uint64_t w = sigma_word<SP, 0>();
            if constexpr (SP::R > 16) {
                sfor<(SP::R + 15) / 16 - 1>([&](auto W) {
                    constexpr int ww = decltype(W)::value + 1;
                    if ((q >> 4) == (unsigned)ww) w = sigma_word<SP, ww>();
                });
            }
            j = (int)((w >> (4 * (q & 15u))) & 15u);
        }
    }
    f.piece = j;
    f.base = base;
    f.in_range = ok;
    return f;
}

// element offset (relative to Fold::base) of stencil site M of piece J: one delta per slot with
// a nonzero offset
template <class SP, int J, int M>
__device__ __forceinline__ int site_offset(const Fold<SP::S> &f)
{
    int off = 0;
    sfor<SP::S>([&](auto A) {
        constexpr int g = SP::SITE[J][M][decltype(A)::value];
        static_assert(g >= -2 && g <= 2, "stencil offsets lie within two sites of the cell");
        if constexpr (g != 0) off += f.sl[A].d[delta_index(g)];
    });
    return off;
}

// gradient back through the fold: d/dx_ax += sign * d/dy'_slot, for each original axis the one
// slot that came from it
template <int S>
__device__ __forceinline__ void unfold_grad(const Fold<S> &f, const float (&gy)[S], float (&grad)[S])
{
    float gs[S];
    sfor<S>([&](auto A) { gs[A] = (f.sl[A].sg < 0) ? -gy[A] : gy[A]; });
    sfor<S>([&](auto B) {
        constexpr int b = decltype(B)::value;
        float g = gs[S - 1];
        sfor<S - 1>([&](auto A) {
            constexpr int a = S - 2 - decltype(A)::value;
            if (f.sl[a].ax == b) g = gs[a];
        });
        grad[b] += g;
    });
}

// steps 4-5 for piece J: accumulate f (and grad f if GRAD) into the query's sums
template <class SP, int J, bool GRAD>
__device__ __forceinline__ void eval_piece_c(const Fold<SP::S> &f, const float (&c)[SP::NS[J]], float &val,
                                             float (&grad)[SP::S]);

template <class SP, int J, bool GRAD, class CT>
__device__ __forceinline__ void eval_piece(const Fold<SP::S> &f, const DevVol<CT> &v, float &val, float (&grad)[SP::S])
{
    constexpr int NS = SP::NS[J];
    const CT *cb = v.c + f.base;
    float c[NS];
    sfor<NS>([&](auto Mi) { c[Mi] = load_coef<CT>(cb + site_offset<SP, J, decltype(Mi)::value>(f)); });
    eval_piece_c<SP, J, GRAD>(f, c, val, grad);
}

// steps 4-5 for piece J on its gathered coefficients c
template <class SP, int J, bool GRAD>
__device__ __forceinline__ void eval_piece_c(const Fold<SP::S> &f, const float (&c)[SP::NS[J]], float &val,
                                             float (&grad)[SP::S])
{
    constexpr int S = SP::S;
    constexpr int NS = SP::NS[J];
    constexpr int NM = SP::NMON;
    float t[S];
    sfor<S>([&](auto A) {
        constexpr float an = SP::ANCHOR[J][decltype(A)::value];
        t[A] = f.t[A] - an;
    });
    constexpr int DEG = SP::DEG;
    VG<S> r;
    if constexpr (NM > 120) {
        // large monomial spaces: Horner in t_1 over blocks P_k(t_2..t_s) (k = DEG .. 0), block k's
        // coefficients formed (b = A_j c restricted to the block) just before they are used
        if constexpr (!GRAD) {
            float acc = 0.0f;
            sfor<DEG + 1>([&](auto I) {
                constexpr int k = DEG - decltype(I)::value;
                constexpr int NMB = nmon(S - 1, DEG - k);
                float bb[NMB];
                sfor<NMB>([&](auto Z) { bb[Z] = 0.0f; });
                accumulate<NS, NMB>(bb, c, typename SP::template NZB<J, k>{});
                const float inner = horner<S, S - 1, DEG - k, 0, NMB>(bb, t);
                if constexpr (k == DEG) acc = inner;
                else acc = fmaf(acc, t[0], inner);
            });
            val += acc;
            return;
        } else {
            sfor<DEG + 1>([&](auto I) {
                constexpr int k = DEG - decltype(I)::value;
                constexpr int NMB = nmon(S - 1, DEG - k);
                float bb[NMB];
                sfor<NMB>([&](auto Z) { bb[Z] = 0.0f; });
                accumulate<NS, NMB>(bb, c, typename SP::template NZB<J, k>{});
                const VG<S - 1> p = horner_grad<S, S - 1, DEG - k, 0, NMB>(bb, t);
                if constexpr (k == DEG) {
                    r.v = p.v;
                    r.g[0] = 0.0f;
                    sfor<S - 1>([&](auto A) { r.g[1 + A] = p.g[A]; });
                } else {
                    if constexpr (k == DEG - 1) r.g[0] = r.v;        // d/dt_1 of the leading block
                    else r.g[0] = fmaf(r.g[0], t[0], r.v);
                    r.v = fmaf(r.v, t[0], p.v);
                    sfor<S - 1>([&](auto A) { r.g[1 + A] = fmaf(r.g[1 + A], t[0], p.g[A]); });
                }
            });
        }
    } else {
        // b = A_j c for every monomial, then nested Horner
        float b[NM];
        sfor<NM>([&](auto A) { b[A] = 0.0f; });
        accumulate<NS, NM>(b, c, typename SP::template NZL<J>{});
        if constexpr (!GRAD) {
            val += horner<S, S, DEG, 0, NM>(b, t);
            return;
        } else {
            r = horner_grad<S, S, DEG, 0, NM>(b, t);
        }
    }
    if constexpr (GRAD) {
        val += r.v;
        unfold_grad<S>(f, r.g, grad);
    }
}

// steps 4-5 for the run-time piece j from the dense tables (splines with SP::DENSE): one loop over
// the piece's stencil sites gathers c_m and adds c_m A_j[:, m] (uniform float4 loads) to b, so the
// pieces share one small copy of the code.  b accumulates over the sites in the same order as
// eval_piece and a zero entry leaves it unchanged, so both give the same sums.
template <class SP, bool GRAD, class CT>
__device__ __forceinline__ void eval_piece_dense(const Fold<SP::S> &f, const DevVol<CT> &v, int j, float &val,
                                                 float (&grad)[SP::S])
{
    constexpr int S = SP::S;
    constexpr int NM = SP::NMON;
    constexpr int NM4 = (NM + 3) / 4;
    static_assert(NM <= 120, "the dense path evaluates b for all monomials at once");
    const CT *cb = v.c + f.base;
    const float4 *A = SP::dense_a(j);
    const signed char *g = SP::dense_site(j);
    const int ns = SP::dense_ns(j);
    float b[NM];
    sfor<NM>([&](auto Z) { b[Z] = 0.0f; });
#pragma unroll 1
    for (int m = 0; m < ns; ++m) {
        int off = 0;
        sfor<S>([&](auto Ax) {
            // the brick geometry of the slot's axis, selected without dynamic indexing
            const int ax = f.sl[Ax].ax;
            int lb = v.L.lb[0], bs = v.L.bstride[0], wt = v.L.wt[0];
            sfor<S - 1>([&](auto B) {
                constexpr int b = 1 + decltype(B)::value;
                if (ax == b) {
                    lb = v.L.lb[b];
                    bs = v.L.bstride[b];
                    wt = v.L.wt[b];
                }
            });
            off += slot_term_rt(f.sl[Ax], (int)__ldg(g + m * S + Ax), lb, bs, wt);
        });
        const float cm = load_coef<CT>(cb + off);
        sfor<NM4>([&](auto Q) {
            constexpr int q = decltype(Q)::value;
            const float4 a4 = __ldg(A + m * NM4 + q);
            b[4 * q] = fmaf(a4.x, cm, b[4 * q]);
            if constexpr (4 * q + 1 < NM) b[4 * q + 1] = fmaf(a4.y, cm, b[4 * q + 1]);
            if constexpr (4 * q + 2 < NM) b[4 * q + 2] = fmaf(a4.z, cm, b[4 * q + 2]);
            if constexpr (4 * q + 3 < NM) b[4 * q + 3] = fmaf(a4.w, cm, b[4 * q + 3]);
        });
    }
    const float *an = SP::dense_anchor(j);
    float t[S];
    sfor<S>([&](auto Ax) { t[Ax] = f.t[Ax] - __ldg(an + Ax); });
    constexpr int DEG = SP::DEG;
    if constexpr (!GRAD) {
        val += horner<S, S, DEG, 0, NM>(b, t);
    } else {
        const VG<S> r = horner_grad<S, S, DEG, 0, NM>(b, t);
        val += r.v;
        unfold_grad<S>(f, r.g, grad);
    }
}

// true when stencil slot M lies at the same offset in every piece that has it (then no per-piece
// select is needed for its address)
template <class SP, int M>
constexpr bool slot_shared()
{
    bool same = M < SP::NS[0];
    for (int j = 1; j < SP::K && same; ++j)
        for (int a = 0; a < SP::S && M < SP::NS[j]; ++a) same = same && SP::SITE[j][M][a] == SP::SITE[0][M][a];
    return same;
}

// steps 4-5 for the run-time piece j of a query whose warp may hold several pieces.  The pieces
// share one monomial space, so only b = A_j c differs in code between them: the site offsets and
// anchors are selected per piece, the coefficient loads, the Horner evaluation and the unfold of
// the gradient run once for every lane, and only the accumulation of b branches.  b accumulates
// each piece's nonzeros in the same order as eval_piece, so both give the same sums.
template <class SP, bool GRAD, class CT>
__device__ __forceinline__ void eval_piece_shared(const Fold<SP::S> &f, const DevVol<CT> &v, float &val,
                                                  float (&grad)[SP::S])
{
    constexpr int S = SP::S;
    constexpr int NM = SP::NMON;
    constexpr int NSM = SP::NSMAX;
    const int j = f.piece;
    const CT *cb = v.c + f.base;
    float c[NSM];
    sfor<NSM>([&](auto Mi) {
        constexpr int m = decltype(Mi)::value;
        // a slot that piece j lacks reads the cell's own site (in range, usually a hit); its value
        // is not used
        int off = 0;
        if constexpr (slot_shared<SP, m>()) {
            off = site_offset<SP, 0, m>(f);
        } else {
            sfor<SP::K>([&](auto Jc) {
                constexpr int J = decltype(Jc)::value;
                if constexpr (m < SP::NS[J]) {
                    if (j == J) off = site_offset<SP, J, m>(f);
                }
            });
        }
        c[m] = load_coef<CT>(cb + off);
    });
    float t[S];
    sfor<S>([&](auto A) {
        constexpr float an0 = SP::ANCHOR[0][decltype(A)::value];
        float an = an0;
        sfor<SP::K - 1>([&](auto Jc) {
            constexpr float anj = SP::ANCHOR[decltype(Jc)::value + 1][decltype(A)::value];
            if (j == decltype(Jc)::value + 1) an = anj;
        });
        t[A] = f.t[A] - an;
    });
    float b[NM];
    sfor<NM>([&](auto A) { b[A] = 0.0f; });
    sfor<SP::K>([&](auto Jc) {
        constexpr int J = decltype(Jc)::value;
        if (j == J) accumulate<NSM, NM>(b, c, typename SP::template NZL<J>{});
    });
    if constexpr (!GRAD) {
        val += horner<S, S, SP::DEG, 0, NM>(b, t);
    } else {
        const VG<S> r = horner_grad<S, S, SP::DEG, 0, NM>(b, t);
        val += r.v;
        unfold_grad<S>(f, r.g, grad);
    }
}

// one binned item of piece j: the dense path or the piece's unrolled code
template <class SP, bool GRAD, class CT, bool DENSE>
__device__ __forceinline__ void eval_item(const Fold<SP::S> &f, const DevVol<CT> &v, int j, float &val,
                                          float (&grad)[SP::S])
{
    if constexpr (DENSE) {
        eval_piece_dense<SP, GRAD, CT>(f, v, j, val, grad);
    } else {
        sfor<SP::K>([&](auto Jc) {
            if (j == decltype(Jc)::value) eval_piece<SP, decltype(Jc)::value, GRAD, CT>(f, v, val, grad);
        });
    }
}

template <class SP, bool GRAD, class CT>
__device__ __forceinline__ void eval_point(const float (&x)[SP::S], const DevVol<CT> &v, float &val,
                                           float (&grad)[SP::S])
{
    if constexpr (SP::K == 1) {
        // one piece: unroll the coset loop (coset shifts become immediates)
        sfor<SP::M>([&](auto Kc) {
            const auto f = fold_coset<SP, decltype(Kc)::value, CT>(x, v);
            if (f.in_range) eval_piece<SP, 0, GRAD, CT>(f, v, val, grad);
        });
    } else if constexpr (SP::NMON <= 120 && (SP::K <= 6 || SP::NNZMAX <= 100) && SP::M * SP::NNZMAX <= 200) {
        // several small pieces (FCC: 4 cosets x 3 pieces of <= 40 nonzeros): the coset loop
        // unrolled as for one piece, the pieces sharing all code but the accumulation of b
        sfor<SP::M>([&](auto Kc) {
            const auto f = fold_coset<SP, decltype(Kc)::value, CT>(x, v);
            if (f.in_range) eval_piece_shared<SP, GRAD, CT>(f, v, val, grad);
        });
    } else {
        // several pieces: run-time coset loop; the pieces share all code but the accumulation of
        // b (monomial spaces up to 120; up to six pieces, or more with small A_j), else one copy of
        // each piece's code (many large pieces: the per-piece address selects would cost more
        // than the shared code saves)
#pragma unroll 1
        for (int k = 0; k < SP::M; ++k) {
            const auto f = fold_coset<SP, -1, CT>(x, v, k);
            if (f.in_range) {
                if constexpr (SP::NMON <= 120 && (SP::K <= 6 || SP::NNZMAX <= 100)) {
                    eval_piece_shared<SP, GRAD, CT>(f, v, val, grad);
                } else {
                    sfor<SP::K>([&](auto Jc) {
                        if (f.piece == decltype(Jc)::value)
                            eval_piece<SP, decltype(Jc)::value, GRAD, CT>(f, v, val, grad);
                    });
                }
            }
        }
    }
}

// MODE 0: out = f.  MODE 1: out = f (if out), grad = grad f.  MODE 2: grad = gout * grad f.
// MINB: resident CTAs per SM the register allocation must allow (1: no bound)
template <class SP, class CT, int MODE, int MINB = 1>
__global__ void __launch_bounds__(128, MINB) k_eval(const float *__restrict__ pts, int64_t n, DevVol<CT> v,
                                              float *__restrict__ out, float *__restrict__ grad,
                                              const float *__restrict__ gout)
{
    constexpr int S = SP::S;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float x[S];
    bool finite = true;
    sfor<S>([&](auto A) {
        x[A] = pts[q * S + A];
        finite &= isfinite(x[A]);
    });
    float val = 0.0f;
    float g[S];
    sfor<S>([&](auto A) { g[A] = 0.0f; });
    if (finite) {
        eval_point<SP, MODE != 0, CT>(x, v, val, g);
    } else {
        val = __int_as_float(0x7fc00000);
        sfor<S>([&](auto A) { g[A] = val; });
    }
    if constexpr (MODE == 0) {
        out[q] = val;
    } else if constexpr (MODE == 1) {
        if (out) out[q] = val;
        sfor<S>([&](auto A) { grad[q * S + A] = g[A]; });
    } else {
        const float w = gout[q];
        sfor<S>([&](auto A) { grad[q * S + A] = w * g[A]; });
    }
}

// Warp-cooperative gathers for one-piece splines (the random-query form of k_eval).  A lane
// folds its query (steps 1-3) and writes the element offsets of its T = M x NS stencil sites to
// its row of a per-warp shared-memory table (T <= 32); the warp then fetches the sites of one
// query per load instruction (lane l: site l), writing each value over its offset, and each lane
// reads its own row back for steps 4-5.  One load instruction then asks
// for the sectors of one compact stencil, so an L1 -> L2 request carries all the sectors the
// query needs in one 128-byte line (BCC quintic: 8.9 lines for 12.5 sectors per query), where a
// load of 32 different queries makes one request per sector.  Sums in the order of k_eval: the
// same results bit for bit.  Every lane of a warp takes part (lanes without a query fetch offset
// 0), so the kernel has no early return.  A warp whose queries lie within 8 cells per axis
// (spatially sorted queries: their sectors are L1 hits anyway) skips the table and runs k_eval's
// per-lane gathers instead, without the table's shared-memory traffic.
constexpr int kCoopCoherentCells = 7;   // coset-0 cell index range per axis of a coherent warp

// the table path of k_eval_coop: steps 1-3 for every coset, the offsets to the lane's row, the
// warp's rounds of gathers, steps 4-5 from the row (warp-synchronous: every lane of the warp).
// Row q holds its 32 words in 16-byte chunks permuted by q mod 8 (chunk c at c ^ (q & 7)): a lane
// writes and reads its row with 16-byte accesses and a round reads and writes one row across the
// warp, both without bank conflicts.
template <class SP, bool GRAD, class CT>
__device__ __forceinline__ void eval_coop_gather(const float (&x)[SP::S], bool finite, const DevVol<CT> &v, int *wt,
                                                 int lane, float &val, float (&g)[SP::S])
{
    constexpr int S = SP::S, M = SP::M, NS = SP::NS[0], T = M * NS;
    static_assert(T <= 32, "one round of loads per query");
    int4 *const row = reinterpret_cast<int4 *>(wt + lane * 32);
    const int sw = lane & 7;
    Fold<S> f[M];
    bool use[M];
    int o[32];
    sfor<32>([&](auto Mi) { o[Mi] = 0; });
    sfor<M>([&](auto Kc) {
        constexpr int K = decltype(Kc)::value;
        f[K] = fold_coset<SP, K, CT>(x, v);
        use[K] = finite && f[K].in_range;
        sfor<NS>([&](auto Mi) {
            constexpr int m = decltype(Mi)::value;
            o[K * NS + m] = use[K] ? f[K].base + site_offset<SP, 0, m>(f[K]) : 0;
        });
    });
    sfor<8>([&](auto Cc) {
        constexpr int c = decltype(Cc)::value;
        row[c ^ sw] = make_int4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]);
    });
    __syncwarp();
    // round r: the sites of the warp's query r, lane l taking site l.  All offsets are read
    // before any value is written back, so the 32 loads are in flight together.
    if (lane < T) {
        // the 8 column positions of lane l (rows r and r + 8 permute alike)
        int *col[8];
        sfor<8>([&](auto Kc) { col[Kc] = wt + ((lane ^ (decltype(Kc)::value << 2)) & 31); });
        int off[32];
        sfor<32>([&](auto Rc) {
            constexpr int r = decltype(Rc)::value;
            off[r] = col[r & 7][r * 32];
        });
        float cw[32];
        sfor<32>([&](auto Rc) { cw[Rc] = load_coef<CT>(v.c + off[Rc]); });
        sfor<32>([&](auto Rc) {
            constexpr int r = decltype(Rc)::value;
            col[r & 7][r * 32] = __float_as_int(cw[r]);
        });
    }
    __syncwarp();
    float cv[32];
    sfor<8>([&](auto Cc) {
        constexpr int c = decltype(Cc)::value;
        const int4 w = row[c ^ sw];
        cv[4 * c] = __int_as_float(w.x);
        cv[4 * c + 1] = __int_as_float(w.y);
        cv[4 * c + 2] = __int_as_float(w.z);
        cv[4 * c + 3] = __int_as_float(w.w);
    });
    sfor<M>([&](auto Kc) {
        constexpr int K = decltype(Kc)::value;
        if (use[K]) {
            float c[NS];
            sfor<NS>([&](auto Mi) { c[Mi] = cv[K * NS + decltype(Mi)::value]; });
            eval_piece_c<SP, 0, GRAD>(f[K], c, val, g);
        }
    });
    __syncwarp();      // the rows are free for the next use
}

template <class SP, class CT, int MODE, int MINB = 1>
__global__ void __launch_bounds__(128, MINB) k_eval_coop(const float *__restrict__ pts, int64_t n, DevVol<CT> v,
                                                         float *__restrict__ out, float *__restrict__ grad,
                                                         const float *__restrict__ gout)
{
    static_assert(SP::K == 1, "cooperative gathers need one stencil for every folded query");
    constexpr int S = SP::S;
    __shared__ __align__(16) int table[4][32 * 32];
    const int lane = threadIdx.x & 31;
    int *const wt = table[threadIdx.x >> 5];
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = q < n;
    float x[S];
    bool finite = live;
    sfor<S>([&](auto A) {
        x[A] = live ? pts[q * S + A] : 0.0f;
        finite &= isfinite(x[A]);
    });
    float val = 0.0f;
    float g[S];
    sfor<S>([&](auto A) { g[A] = 0.0f; });
    // the warp's extent in coset-0 cells (lanes without a finite query are neutral)
    bool coherent = true;
    sfor<S>([&](auto A) {
        const int cell = finite ? __float2int_rd(x[A] * (1.0f / SP::D)) : 0;
        const int lo = __reduce_min_sync(0xffffffffu, finite ? cell : 0x7fffffff);
        const int hi = __reduce_max_sync(0xffffffffu, finite ? cell : -0x7fffffff - 1);
        coherent &= (long long)hi - lo <= kCoopCoherentCells;
    });
    if (coherent) {
        if (finite) eval_point<SP, MODE != 0, CT>(x, v, val, g);
    } else {
        eval_coop_gather<SP, MODE != 0, CT>(x, finite, v, wt, lane, val, g);
    }
    if (!live) return;
    if (!finite) {
        val = __int_as_float(0x7fc00000);
        sfor<S>([&](auto A) { g[A] = val; });
    }
    if constexpr (MODE == 0) {
        out[q] = val;
    } else if constexpr (MODE == 1) {
        if (out) out[q] = val;
        sfor<S>([&](auto A) { grad[q * S + A] = g[A]; });
    } else {
        const float w = gout[q];
        sfor<S>([&](auto A) { grad[q * S + A] = w * g[A]; });
    }
}

// ------------------------------------------------------------------------------------ adjoint

// w_site = sum_mon A[mon][site] mu[mon]; at the last nonzero of a site, scatter it
template <class SP, int J, int NM, int SITE, int MON, float VAL, int FIRST, int SF, int SL>
__device__ __forceinline__ void nz_scatter(const float (&mu)[NM], float &acc, const Fold<SP::S> &f, float *db,
                                           interp_gen::nz<SITE, MON, VAL, FIRST, SF, SL>)
{
    if constexpr (SF) acc = mu[MON] * VAL;
    else acc = fmaf(mu[MON], VAL, acc);
    if constexpr (SL) atomicAdd(db + site_offset<SP, J, SITE>(f), acc);
}
template <class SP, int J, int NM, class... Z>
__device__ __forceinline__ void scatter_all(const float (&mu)[NM], const Fold<SP::S> &f, float *db, interp_gen::nzlist<Z...>)
{
    float acc = 0.0f;
    (nz_scatter<SP, J, NM>(mu, acc, f, db, Z{}), ...);
}

// dpad[site] += gout * phi(x - site) for every stencil site of piece J (padded FP32 layout)
template <class SP, int J>
__device__ __forceinline__ void adjoint_piece(const Fold<SP::S> &f, float *__restrict__ dpad, float w)
{
    constexpr int S = SP::S;
    constexpr int NM = SP::NMON;
    float t[S];
    sfor<S>([&](auto A) {
        constexpr float an = SP::ANCHOR[J][decltype(A)::value];
        t[A] = f.t[A] - an;
    });
    float mu[NM];
    monomials<S, S, SP::DEG, 0, NM>(mu, t, w);     // w * t^alpha
    scatter_all<SP, J, NM>(mu, f, dpad + f.base, typename SP::template NZL<J>{});
}

template <class SP>
__global__ void __launch_bounds__(128) k_adjoint(const float *__restrict__ pts, int64_t n,
                                                 const float *__restrict__ gout, DevVol<float> v,
                                                 float *__restrict__ dpad)
{
    constexpr int S = SP::S;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float x[S];
    bool finite = true;
    sfor<S>([&](auto A) {
        x[A] = pts[q * S + A];
        finite &= isfinite(x[A]);
    });
    const float w = gout[q];
    if (!finite || w == 0.0f) return;
    if constexpr (SP::K == 1) {
        sfor<SP::M>([&](auto Kc) {
            const auto f = fold_coset<SP, decltype(Kc)::value, float>(x, v);
            if (f.in_range) adjoint_piece<SP, 0>(f, dpad, w);
        });
    } else {
#pragma unroll 1
        for (int k = 0; k < SP::M; ++k) {
            const auto f = fold_coset<SP, -1, float>(x, v, k);
            if (f.in_range) {
                sfor<SP::K>([&](auto Jc) {
                    if (f.piece == decltype(Jc)::value) adjoint_piece<SP, decltype(Jc)::value>(f, dpad, w);
                });
            }
        }
    }
}

// ------------------------------------------------------------------------------------ debug indices

template <class SP>
__global__ void k_debug(const float *__restrict__ pts, int64_t n, DevVol<float> v, int32_t *__restrict__ cells,
                        int32_t *__restrict__ piece)
{
    constexpr int S = SP::S;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float x[S];
    sfor<S>([&](auto A) { x[A] = pts[q * S + A]; });
    sfor<SP::M>([&](auto Kc) {
        constexpr int K = decltype(Kc)::value;
        if (cells) {
            sfor<S>([&](auto A) {
                constexpr int a = decltype(A)::value;
                int i;
                float y;
                reduce_axis<SP::D, SP::COSET[K][a]>(x[a], i, y);
                cells[(q * SP::M + K) * S + a] = i;
            });
        }
        if (piece) {
            const auto f = fold_coset<SP, K, float>(x, v);
            piece[q * SP::M + K] = f.piece;
        }
    });
}

}  // namespace ib

// ------------------------------------------------------------------------------------ batched launch

namespace ib {

using ibl::BatchVol;

// evaluate queries [q0, q1) of one volume with spline SP, block-strided
template <class SP>
__device__ __forceinline__ void batch_tile(const BatchVol &bv, int64_t q0, int64_t q1)
{
    constexpr int S = SP::S;
    DevVol<float> v;
    v.c = bv.c;
    v.L = bv.L;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        float x[S];
        bool finite = true;
        sfor<S>([&](auto A) {
            x[A] = bv.pts[q * S + A];
            finite &= isfinite(x[A]);
        });
        float val = 0.0f, g[S];
        if (finite) eval_point<SP, false, float>(x, v, val, g);
        else val = __int_as_float(0x7fc00000);
        bv.out[q] = val;
    }
}

template <class... SPs> struct SplineList {};

template <int I, class SP0, class... SPs>
__device__ __forceinline__ void batch_dispatch(int kind, const BatchVol &bv, int64_t q0, int64_t q1)
{
    if (kind == I) batch_tile<SP0>(bv, q0, q1);
    else if constexpr (sizeof...(SPs) > 0) batch_dispatch<I + 1, SPs...>(kind, bv, q0, q1);
}

// Persistent kernel: every CTA repeatedly claims the next work item (volume, tile) from a
// global counter; the spline is uniform inside a CTA, so the dispatch does not diverge (pieces
// of a multi-piece spline still diverge inside a warp; the 6-piece 4-D spline is therefore
// evaluated by the piece-binned kernel, not here).  Work
// item ids are ordered volume by volume; a CTA finds its volume by binary search over the
// per-volume first-tile prefix.  The counter is zeroed before each launch (a memset node of the
// same graph); the loop ends when the counter passes the total, so it always terminates.
// Five resident CTAs per SM (96 registers, no spills; unbounded it takes 121 and four).
template <class... SPs>
__global__ void __launch_bounds__(128, 5) k_batch(const BatchVol *__restrict__ vols, int nvol, int64_t total_tiles,
                                               unsigned long long *__restrict__ counter)
{
    __shared__ long long item;
    for (;;) {
        if (threadIdx.x == 0) item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = item;
        __syncthreads();
        if (it >= total_tiles) return;
        int lo = 0, hi = nvol - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (vols[mid].first_tile <= it) lo = mid;
            else hi = mid - 1;
        }
        const BatchVol &bv = vols[lo];
        const int64_t q0 = (it - bv.first_tile) * bv.tile;
        const int64_t q1 = q0 + bv.tile < bv.npts ? q0 + bv.tile : bv.npts;
        batch_dispatch<0, SPs...>(bv.kind, bv, q0, q1);
    }
}

}  // namespace ib

// ------------------------------------------------------------------------------------ rays

namespace ib {

// Orthographic rays: pixel (px, py) starts at o = origin + (px+1/2) du + (py+1/2) dv and runs
// along dir; its chord with the box [lo, hi] is split into `steps` equal steps, sampled at the
// step midpoints.  Per pixel: sum over samples of f (and of grad f).  A warp covers an 8 x 4
// block of pixels, so its samples are close together and share coefficient sectors in L1.
using ibl::RayGeom;

// ray of pixel (px, py): origin o, and the entry parameter tmin and step dt of its samples
// inside the box [lo, hi] (sample i at o + (tmin + (i + 1/2) dt) dir); false if it misses the box
__device__ __forceinline__ bool ray_setup(const RayGeom &rg, int px, int py, float (&o)[3], float &tmin, float &dt)
{
    float tmax = 3.0e38f;
    tmin = -3.0e38f;
    sfor<3>([&](auto A) {
        o[A] = rg.origin[A] + ((float)px + 0.5f) * rg.du[A] + ((float)py + 0.5f) * rg.dv[A];
        if (rg.dir[A] != 0.0f) {
            const float inv = 1.0f / rg.dir[A];
            const float t1 = (rg.lo[A] - o[A]) * inv, t2 = (rg.hi[A] - o[A]) * inv;
            tmin = fmaxf(tmin, fminf(t1, t2));
            tmax = fminf(tmax, fmaxf(t1, t2));
        } else if (o[A] < rg.lo[A] || o[A] > rg.hi[A]) {
            tmax = -3.0e38f;                                  // parallel to the slab and outside
        }
    });
    dt = (tmax - tmin) / (float)rg.steps;
    return tmax > tmin;
}

template <class SP, bool GRAD>
__global__ void __launch_bounds__(128) k_rays(RayGeom rg, DevVol<float> v, float *__restrict__ out,
                                              float *__restrict__ pts_out)
{
    static_assert(SP::S == 3, "rays are 3-D");
    // 128 threads = 4 warps; a block covers 16 x 8 pixels, a warp 8 x 4
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int py = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    if (px >= rg.width || py >= rg.height) return;
    float o[3], tmin, dt;
    float val = 0.0f, g[3] = {0.0f, 0.0f, 0.0f};
    const int64_t pix = (int64_t)py * rg.width + px;
    if (ray_setup(rg, px, py, o, tmin, dt)) {
        for (int i = 0; i < rg.steps; ++i) {
            const float t = tmin + ((float)i + 0.5f) * dt;
            float x[3];
            sfor<3>([&](auto A) { x[A] = fmaf(t, rg.dir[A], o[A]); });
            if (pts_out) sfor<3>([&](auto A) { pts_out[(pix * rg.steps + i) * 3 + A] = x[A]; });
            eval_point<SP, GRAD, float>(x, v, val, g);
        }
    } else if (pts_out) {
        for (int i = 0; i < rg.steps; ++i)
            sfor<3>([&](auto A) { pts_out[(pix * rg.steps + i) * 3 + A] = __int_as_float(0x7fc00000); });
    }
    out[pix * (GRAD ? 4 : 1)] = val;
    if constexpr (GRAD) sfor<3>([&](auto A) { out[pix * 4 + 1 + A] = g[A]; });
}

}  // namespace ib

// ------------------------------------------------------------------------------------ piece-binned evaluation

namespace ib {

// A multi-piece spline makes the piece data dependent: a warp whose 32 queries fall in K pieces
// runs all K piece codes.  This kernel takes a tile of T queries x M cosets, classifies every
// (query, coset) item (steps 1-3), sorts the items by piece in shared memory (counting sort),
// then evaluates them in sorted order, so each warp sees one piece except where two pieces'
// runs meet.  Per-(query, coset) results go to shared memory and are summed over the cosets in
// a fixed order, so the output does not depend on the schedule.
template <int S> struct BinRec {
    int base;       // Fold::base
    float t[S];     // folded offset
    unsigned slots; // per slot (5 bits): sign (1), original axis (2), within-brick coordinate (2)
};

template <class SP, class CT>
__device__ __forceinline__ Fold<SP::S> unpack_rec(const BinRec<SP::S> &r, const DevVol<CT> &v)
{
    constexpr int S = SP::S;
    Fold<S> f;
    f.base = r.base;
    f.in_range = true;
    sfor<S>([&](auto A) {
        const unsigned b = (r.slots >> (5 * A)) & 31u;
        Slot &sl = f.sl[A];
        sl.y = r.t[A];
        f.t[A] = r.t[A];
        sl.sg = (b & 1u) ? -1 : 1;
        sl.ax = (int)((b >> 1) & 3u);
        sl.p = (int)(b >> 3);
        // the brick geometry of the slot's axis, selected without dynamic indexing
        int lb = v.L.lb[0], bs = v.L.bstride[0], wt = v.L.wt[0];
        sfor<S - 1>([&](auto B) {
            constexpr int ax = 1 + decltype(B)::value;
            if (sl.ax == ax) {
                lb = v.L.lb[ax];
                bs = v.L.bstride[ax];
                wt = v.L.wt[ax];
            }
        });
        slot_deltas_rt<SP>(sl, lb, bs, wt);
    });
    return f;
}

// shared memory of k_eval_binned for a tile of T queries
template <class SP, int MODE, int T>
constexpr size_t binned_smem_bytes()
{
    constexpr int NI = T * SP::M;
    constexpr int NV = MODE != 0 ? SP::S + 1 : 1;
    return (size_t)NI * (sizeof(BinRec<SP::S>) + NV * sizeof(float) + 2 * sizeof(unsigned short) + 1) + 64;
}

// classify the tile's (query, coset) items and counting-sort them by piece in shared memory:
// on return perm[0 .. start[K]) lists the live items in piece order (ends with a barrier).
// src(ql, x) fills the coordinates of local query ql and returns false for a query that is
// absent or not finite (its items are dropped).
template <class SP, class CT, int T, class Src>
__device__ __forceinline__ void bin_tile_src(Src &&src, const DevVol<CT> &v, BinRec<SP::S> *rec,
                                             unsigned short *perm, unsigned short *rank, signed char *rpiece,
                                             int *cnt, int *start)
{
    constexpr int S = SP::S, M = SP::M, K = SP::K, NI = T * M;
    const int tid = threadIdx.x;
    if (tid < K) cnt[tid] = 0;
    __syncthreads();
    // classify: item i = (query i % T, coset i / T)
    for (int i = tid; i < NI; i += blockDim.x) {
        const int ql = i % T, k = i / T;
        int j = -1;
        float x[S];
        if (src(ql, x)) {
            const Fold<S> f = fold_coset<SP, -1, CT>(x, v, k);
            if (f.in_range) {
                j = f.piece;
                BinRec<S> r;
                r.base = f.base;
                unsigned slots = 0;
                sfor<S>([&](auto A) {
                    r.t[A] = f.t[A];
                    slots |= ((f.sl[A].sg < 0 ? 1u : 0u) | ((unsigned)f.sl[A].ax << 1) | ((unsigned)f.sl[A].p << 3))
                             << (5 * A);
                });
                r.slots = slots;
                rec[i] = r;
                rank[i] = (unsigned short)atomicAdd(&cnt[j], 1);
            }
        }
        rpiece[i] = (signed char)j;
    }
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int j = 0; j < K; ++j) {
            start[j] = s;
            s += cnt[j];
        }
        start[K] = s;
    }
    __syncthreads();
    for (int i = tid; i < NI; i += blockDim.x)
        if (rpiece[i] >= 0) perm[start[rpiece[i]] + rank[i]] = (unsigned short)i;
    __syncthreads();
}

// the same for the tile of T queries starting at q0 of the point array pts (n points)
template <class SP, class CT, int T>
__device__ __forceinline__ void bin_tile(const float *__restrict__ pts, int64_t n, const DevVol<CT> &v, int64_t q0,
                                         BinRec<SP::S> *rec, unsigned short *perm, unsigned short *rank,
                                         signed char *rpiece, int *cnt, int *start)
{
    constexpr int S = SP::S;
    bin_tile_src<SP, CT, T>(
        [&](int ql, float (&x)[S]) {
            const int64_t q = q0 + ql;
            if (q >= n) return false;
            bool finite = true;
            sfor<S>([&](auto A) {
                x[A] = pts[q * S + A];
                finite &= isfinite(x[A]);
            });
            return finite;
        },
        v, rec, perm, rank, rpiece, cnt, start);
}

// T queries per tile, NT threads per CTA.  With NT = 512 and a large tile the CTA fills an SM,
// and its warps walk through the sorted pieces together, so only one or two pieces' code is hot
// in the instruction caches at a time.
template <class SP, class CT, int MODE, int T, int NT, bool DENSE = false>
__global__ void __launch_bounds__(NT) k_eval_binned(const float *__restrict__ pts, int64_t n, DevVol<CT> v,
                                                    float *__restrict__ out, float *__restrict__ grad,
                                                    const float *__restrict__ gout)
{
    constexpr int S = SP::S, M = SP::M, K = SP::K, NI = T * M;
    constexpr bool GRAD = MODE != 0;
    constexpr int NV = GRAD ? S + 1 : 1;            // value (and gradient) per item
    static_assert(NI <= 65535, "item index must fit 16 bits");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BinRec<S> *rec = reinterpret_cast<BinRec<S> *>(smem_raw);
    float *acc = reinterpret_cast<float *>(rec + NI);
    unsigned short *perm = reinterpret_cast<unsigned short *>(acc + NI * NV);
    unsigned short *rank = perm + NI;
    signed char *rpiece = reinterpret_cast<signed char *>(rank + NI);
    __shared__ int cnt[K], start[K + 1];
    const int tid = threadIdx.x;
    const int64_t q0 = (int64_t)blockIdx.x * T;
    for (int i = tid; i < NI * NV; i += blockDim.x) acc[i] = 0.0f;
    bin_tile<SP, CT, T>(pts, n, v, q0, rec, perm, rank, rpiece, cnt, start);
    // evaluate in piece order: consecutive lanes take consecutive sorted items
    const int total = start[K];
    for (int p = tid; p < total; p += blockDim.x) {
        const int i = perm[p];
        const int j = rpiece[i];
        const Fold<S> f = unpack_rec<SP, CT>(rec[i], v);
        float val = 0.0f, g[S];
        sfor<S>([&](auto A) { g[A] = 0.0f; });
        eval_item<SP, GRAD, CT, DENSE>(f, v, j, val, g);
        acc[i * NV] = val;
        if constexpr (GRAD) sfor<S>([&](auto A) { acc[i * NV + 1 + A] = g[A]; });
    }
    __syncthreads();
    // sum over cosets in coset order and write out
    for (int ql = tid; ql < T; ql += blockDim.x) {
        const int64_t q = q0 + ql;
        if (q >= n) break;
        bool finite = true;
        sfor<S>([&](auto A) { finite &= isfinite(pts[q * S + A]); });
        float val = 0.0f, g[S];
        sfor<S>([&](auto A) { g[A] = 0.0f; });
        sfor<M>([&](auto Kc) {
            const int i = Kc * T + ql;
            val += acc[i * NV];
            if constexpr (GRAD) sfor<S>([&](auto A) { g[A] += acc[i * NV + 1 + A]; });
        });
        if (!finite) {
            val = __int_as_float(0x7fc00000);
            sfor<S>([&](auto A) { g[A] = val; });
        }
        if constexpr (MODE == 0) {
            out[q] = val;
        } else if constexpr (MODE == 1) {
            if (out) out[q] = val;
            sfor<S>([&](auto A) { grad[q * S + A] = g[A]; });
        } else {
            const float w = gout[q];
            sfor<S>([&](auto A) { grad[q * S + A] = w * g[A]; });
        }
    }
}

// adjoint of a multi-piece spline, piece-binned like k_eval_binned: after the sort each warp
// scatters one piece's contributions (global atomics into the padded buffer)
template <class SP, int T, int NT>
__global__ void __launch_bounds__(NT) k_adjoint_binned(const float *__restrict__ pts, int64_t n,
                                                       const float *__restrict__ gout, DevVol<float> v,
                                                       float *__restrict__ dpad)
{
    constexpr int S = SP::S, M = SP::M, K = SP::K, NI = T * M;
    static_assert(NI <= 65535, "item index must fit 16 bits");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BinRec<S> *rec = reinterpret_cast<BinRec<S> *>(smem_raw);
    unsigned short *perm = reinterpret_cast<unsigned short *>(rec + NI);
    unsigned short *rank = perm + NI;
    signed char *rpiece = reinterpret_cast<signed char *>(rank + NI);
    __shared__ int cnt[K], start[K + 1];
    const int64_t q0 = (int64_t)blockIdx.x * T;
    bin_tile<SP, float, T>(pts, n, v, q0, rec, perm, rank, rpiece, cnt, start);
    const int total = start[K];
    for (int p = threadIdx.x; p < total; p += blockDim.x) {
        const int i = perm[p];
        const float w = gout[q0 + i % T];
        if (w == 0.0f) continue;
        const int j = rpiece[i];
        const Fold<S> f = unpack_rec<SP, float>(rec[i], v);
        sfor<K>([&](auto Jc) {
            if (j == decltype(Jc)::value) adjoint_piece<SP, decltype(Jc)::value>(f, dpad, w);
        });
    }
}

// rays of a multi-piece spline, piece-binned: a tile holds RT = T / steps whole rays (the host
// launches it only for steps <= T); the samples come from the ray geometry, are classified and
// sorted by piece as in k_eval_binned, evaluated in piece order, and summed per ray in step order
// and coset order -- the order of k_rays, so both kernels return the same sums.  One CTA per tile.
template <class SP, bool GRAD, int T, int NT, bool DENSE = false>
__global__ void __launch_bounds__(NT) k_rays_binned(RayGeom rg, DevVol<float> v, float *__restrict__ out,
                                                    float *__restrict__ pts_out)
{
    static_assert(SP::S == 3, "rays are 3-D");
    constexpr int S = 3, M = SP::M, K = SP::K, NI = T * M;
    constexpr int NV = GRAD ? S + 1 : 1;
    static_assert(NI <= 65535, "item index must fit 16 bits");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BinRec<S> *rec = reinterpret_cast<BinRec<S> *>(smem_raw);
    float *acc = reinterpret_cast<float *>(rec + NI);
    unsigned short *perm = reinterpret_cast<unsigned short *>(acc + NI * NV);
    unsigned short *rank = perm + NI;
    signed char *rpiece = reinterpret_cast<signed char *>(rank + NI);
    __shared__ int cnt[K], start[K + 1];
    const int tid = threadIdx.x;
    const int steps = rg.steps;
    const int RT = T / steps;
    const int64_t npix = (int64_t)rg.width * rg.height;
    const int64_t r0 = (int64_t)blockIdx.x * RT;
    for (int i = tid; i < NI * NV; i += blockDim.x) acc[i] = 0.0f;
    // sample ql of the tile: ray r0 + ql / steps, step ql % steps
    auto sample = [&](int ql, float (&x)[S]) {
        const int rl = ql / steps, i = ql - rl * steps;
        const int64_t pix = r0 + rl;
        if (rl >= RT || pix >= npix) return false;
        float o[3], tmin, dt;
        if (!ray_setup(rg, (int)(pix % rg.width), (int)(pix / rg.width), o, tmin, dt)) return false;
        const float t = tmin + ((float)i + 0.5f) * dt;
        sfor<S>([&](auto A) { x[A] = fmaf(t, rg.dir[A], o[A]); });
        return true;
    };
    if (pts_out) {
        for (int ql = tid; ql < RT * steps; ql += blockDim.x) {
            const int64_t q = r0 * steps + ql;
            if (q >= npix * steps) break;
            float x[S];
            if (!sample(ql, x)) sfor<S>([&](auto A) { x[A] = __int_as_float(0x7fc00000); });
            sfor<S>([&](auto A) { pts_out[q * S + A] = x[A]; });
        }
    }
    bin_tile_src<SP, float, T>(sample, v, rec, perm, rank, rpiece, cnt, start);
    const int total = start[K];
    for (int p = tid; p < total; p += blockDim.x) {
        const int i = perm[p];
        const int j = rpiece[i];
        const Fold<S> f = unpack_rec<SP, float>(rec[i], v);
        float val = 0.0f, g[S];
        sfor<S>([&](auto A) { g[A] = 0.0f; });
        eval_item<SP, GRAD, float, DENSE>(f, v, j, val, g);
        acc[i * NV] = val;
        if constexpr (GRAD) sfor<S>([&](auto A) { acc[i * NV + 1 + A] = g[A]; });
    }
    __syncthreads();
    for (int rl = tid; rl < RT; rl += blockDim.x) {
        const int64_t pix = r0 + rl;
        if (pix >= npix) break;
        float val = 0.0f, g[S] = {0.0f, 0.0f, 0.0f};
        for (int i = 0; i < steps; ++i) {
            sfor<M>([&](auto Kc) {
                const int it = Kc * T + rl * steps + i;
                if (rpiece[it] >= 0) {
                    val += acc[it * NV];
                    if constexpr (GRAD) sfor<S>([&](auto A) { g[A] += acc[it * NV + 1 + A]; });
                }
            });
        }
        out[pix * (GRAD ? 4 : 1)] = val;
        if constexpr (GRAD) sfor<S>([&](auto A) { out[pix * 4 + 1 + A] = g[A]; });
    }
}

template <class SP, int T>
constexpr size_t binned_adjoint_smem_bytes()
{
    constexpr int NI = T * SP::M;
    return (size_t)NI * (sizeof(BinRec<SP::S>) + 2 * sizeof(unsigned short) + 1) + 64;
}

}  // namespace ib

// ------------------------------------------------------------------------------------ spatial sort

namespace ib {

// Bin of a query for the spatial sort: the padded cell index of coset 0, clamped to the array,
// divided by 2^BB per axis, the bin coordinates interleaved bit by bit (Morton / Z order), so
// queries that are close in space get close keys and a run of sorted queries covers a compact box.
template <class SP>
__device__ __forceinline__ unsigned sort_key(const float (&x)[SP::S], const ibl::Layout &L, int bb, int bits)
{
    constexpr int S = SP::S;
    unsigned bin[S];
    sfor<S>([&](auto A) {
        constexpr int a = decltype(A)::value;
        int i;
        float y;
        reduce_axis<SP::D, SP::COSET[0][a]>(x[a], i, y);
        int P = i + L.pad;
        P = P < 0 ? 0 : (P > L.pdims[a] - 1 ? L.pdims[a] - 1 : P);
        bin[a] = (unsigned)P >> bb;
    });
    unsigned key = 0;
    for (int b = 0; b < bits; ++b)
        sfor<S>([&](auto A) { key |= ((bin[A] >> b) & 1u) << (b * S + A); });
    return key;
}

// in-place exclusive prefix sum of n counters, one CTA of NT threads (n up to a few million);
// a template so that every translation unit including this header has its own copy
template <int NT>
__global__ void __launch_bounds__(NT) k_scan_exclusive(unsigned *__restrict__ a, int n)
{
    static_assert(NT == 1024, "one CTA of 1024 threads");
    __shared__ unsigned part[1024];
    const int per = (n + 1023) / 1024;
    const int beg = threadIdx.x * per;
    const int end = beg + per < n ? beg + per : n;
    unsigned s = 0;
    for (int i = beg; i < end; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {          // inclusive Hillis-Steele scan
        const unsigned v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = beg; i < end; ++i) {
        const unsigned t = a[i];
        a[i] = run;
        run += t;
    }
}

// Parallel exclusive prefix sum of n counters in three launches: per-block sums of 4096
// elements, an exclusive scan of those sums (k_scan_exclusive, one CTA), then a scan of every
// block offset by its sum.  Templates, like k_scan_exclusive, so every unit has its own copy.
constexpr int kScanBlock = 4096;

template <int NT>
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned *part, unsigned &total)
{
    part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < NT; off <<= 1) {
        const unsigned u = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += u;
        __syncthreads();
    }
    total = part[NT - 1];
    const unsigned ex = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    __syncthreads();
    return ex;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_scan_block_sums(const unsigned *__restrict__ a, int n, unsigned *__restrict__ sums)
{
    static_assert(NT * 4 == kScanBlock, "4 elements per thread");
    __shared__ unsigned part[NT];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
    unsigned v = 0;
    for (int i = 0; i < 4; ++i) v += base + i < n ? a[base + i] : 0u;
    unsigned total;
    block_exclusive_scan<NT>(v, part, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_scan_apply(unsigned *__restrict__ a, int n, const unsigned *__restrict__ sums)
{
    __shared__ unsigned part[NT];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
    unsigned v[4], s = 0;
    for (int i = 0; i < 4; ++i) {
        v[i] = base + i < n ? a[base + i] : 0u;
        s += v[i];
    }
    unsigned total;
    unsigned run = block_exclusive_scan<NT>(s, part, total) + sums[blockIdx.x];
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) a[base + i] = run;
        run += v[i];
    }
}

template <class SP>
__global__ void k_sort_count(const float *__restrict__ pts, int64_t n, ibl::Layout L, int bb, int bits,
                             unsigned *__restrict__ counts)
{
    constexpr int S = SP::S;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        float x[S];
        sfor<S>([&](auto A) {
            const float v = pts[q * S + A];
            x[A] = isfinite(v) ? v : 0.0f;             // non-finite queries go to some bin
        });
        atomicAdd(&counts[sort_key<SP>(x, L, bb, bits)], 1u);
    }
}

template <class SP>
__global__ void k_sort_scatter(const float *__restrict__ pts, int64_t n, ibl::Layout L, int bb, int bits,
                               unsigned *__restrict__ cursor, int32_t *__restrict__ perm, float *__restrict__ pts_out)
{
    constexpr int S = SP::S;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        float x[S], xr[S];
        sfor<S>([&](auto A) {
            xr[A] = pts[q * S + A];
            x[A] = isfinite(xr[A]) ? xr[A] : 0.0f;
        });
        const unsigned pos = atomicAdd(&cursor[sort_key<SP>(x, L, bb, bits)], 1u);
        if (perm) perm[pos] = (int32_t)q;
        if (pts_out) sfor<S>([&](auto A) { pts_out[(int64_t)pos * S + A] = xr[A]; });
    }
}

// ------------------------------------------------------------------------------------ privatised adjoint

// w_site = sum_mon A[mon][site] mu[mon]; at the last nonzero of a site, add it to the CTA's
// shared-memory copy of the box around its queries (local linear offsets)
template <class SP, int J, int NM, int SITE, int MON, float VAL, int FIRST, int SF, int SL>
__device__ __forceinline__ void nz_scatter_local(const float (&mu)[NM], float &acc, const int (&lss)[SP::S], int lbase,
                                                 float *sacc, interp_gen::nz<SITE, MON, VAL, FIRST, SF, SL>)
{
    if constexpr (SF) acc = mu[MON] * VAL;
    else acc = fmaf(mu[MON], VAL, acc);
    if constexpr (SL) {
        int off = lbase;
        sfor<SP::S>([&](auto A) {
            constexpr int g = SP::SITE[J][SITE][decltype(A)::value];
            if constexpr (g != 0) off += g * lss[A];
        });
        atomicAdd(sacc + off, acc);
    }
}
template <class SP, int J, int NM, class... Z>
__device__ __forceinline__ void scatter_local_all(const float (&mu)[NM], const int (&lss)[SP::S], int lbase, float *sacc,
                                                  interp_gen::nzlist<Z...>)
{
    float acc = 0.0f;
    (nz_scatter_local<SP, J, NM>(mu, acc, lss, lbase, sacc, Z{}), ...);
}

template <class SP, int J>
__device__ __forceinline__ void adjoint_piece_local(const Fold<SP::S> &f, const int (&lss)[SP::S], int lbase,
                                                    float *sacc, float w)
{
    constexpr int S = SP::S;
    constexpr int NM = SP::NMON;
    float t[S];
    sfor<S>([&](auto A) {
        constexpr float an = SP::ANCHOR[J][decltype(A)::value];
        t[A] = f.t[A] - an;
    });
    float mu[NM];
    monomials<S, S, SP::DEG, 0, NM>(mu, t, w);
    scatter_local_all<SP, J, NM>(mu, lss, lbase, sacc, typename SP::template NZL<J>{});
}

// Adjoint over chunks of CH queries per CTA.  Each CTA first finds the padded-cell bounding box
// of its queries (all cosets); if the box plus the stencil halo fits in shared memory -- it does
// when the queries are sorted spatially -- the contributions are summed there with shared-memory
// atomics and added to the global buffer once per site; otherwise every contribution goes
// straight to the global buffer (unsorted queries).
constexpr int kAdjChunk = 1024;
constexpr int kAdjSmemFloats = 6144;

template <class SP>
__global__ void __launch_bounds__(256, 2) k_adjoint_priv(const float *__restrict__ pts, int64_t n,
                                                      const float *__restrict__ gout, DevVol<float> v,
                                                      float *__restrict__ dpad)
{
    constexpr int S = SP::S, M = SP::M, H = SP::HALO;
    __shared__ float sacc[kAdjSmemFloats];
    __shared__ int bmin[S], bmax[S];
    const int64_t c0 = (int64_t)blockIdx.x * kAdjChunk;
    const int64_t c1 = c0 + kAdjChunk < n ? c0 + kAdjChunk : n;
    if (threadIdx.x < S) {
        bmin[threadIdx.x] = 0x7fffffff;
        bmax[threadIdx.x] = -0x7fffffff;
    }
    __syncthreads();
    // pass 1: bounding box of the padded cell indices (every coset) of the chunk's live queries
    for (int64_t q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
        float x[S];
        bool ok = gout[q] != 0.0f;
        sfor<S>([&](auto A) {
            x[A] = pts[q * S + A];
            ok &= isfinite(x[A]);
        });
        if (!ok) continue;
        sfor<M>([&](auto Kc) {
            constexpr int K = decltype(Kc)::value;
            int P[S];
            bool in = true;
            sfor<S>([&](auto A) {
                constexpr int a = decltype(A)::value;
                float y;
                int i;
                reduce_axis<SP::D, SP::COSET[K][a]>(x[a], i, y);
                in &= (unsigned)(i + H) < (unsigned)(v.L.n[a] + 2 * H);
                P[a] = i + 2 * H;
            });
            if (in)
                sfor<S>([&](auto A) {
                    atomicMin(&bmin[A], P[A]);
                    atomicMax(&bmax[A], P[A]);
                });
        });
    }
    __syncthreads();
    int ld[S], lstride[S];
    int vol = 1;
    bool empty = false;
    for (int a = S - 1; a >= 0; --a) {
        empty |= bmax[a] < bmin[a];
        ld[a] = bmax[a] - bmin[a] + 1 + 2 * H;
        lstride[a] = vol;
        vol = (vol < (1 << 24) && ld[a] > 0) ? vol * ld[a] : (1 << 24);
    }
    if (empty) return;
    const bool priv = (int64_t)vol * M <= kAdjSmemFloats;
    if (priv) {
        for (int i = threadIdx.x; i < vol * M; i += blockDim.x) sacc[i] = 0.0f;
        __syncthreads();
    }
    // pass 2: the contributions
    for (int64_t q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
        float x[S];
        bool finite = true;
        sfor<S>([&](auto A) {
            x[A] = pts[q * S + A];
            finite &= isfinite(x[A]);
        });
        const float w = gout[q];
        if (!finite || w == 0.0f) continue;
        sfor<M>([&](auto Kc) {
            constexpr int K = decltype(Kc)::value;
            const auto f = fold_coset<SP, K, float>(x, v);
            if (!f.in_range) return;
            if (priv) {
                // local offset of the cell's site and signed local strides per folded slot
                int P[S];
                sfor<S>([&](auto A) {
                    constexpr int a = decltype(A)::value;
                    float y;
                    int i;
                    reduce_axis<SP::D, SP::COSET[K][a]>(x[a], i, y);
                    P[a] = i + 2 * H;
                });
                int lbase = K * vol, lss[S];
                sfor<S>([&](auto A) {
                    lbase += (P[A] - bmin[A] + H) * lstride[A];
                    int st = lstride[0];
                    sfor<S - 1>([&](auto B) {
                        if (f.sl[A].ax == 1 + decltype(B)::value) st = lstride[1 + decltype(B)::value];
                    });
                    lss[A] = f.sl[A].sg * st;
                });
                sfor<SP::K>([&](auto Jc) {
                    if (f.piece == decltype(Jc)::value) adjoint_piece_local<SP, decltype(Jc)::value>(f, lss, lbase, sacc, w);
                });
            } else {
                sfor<SP::K>([&](auto Jc) {
                    if (f.piece == decltype(Jc)::value) adjoint_piece<SP, decltype(Jc)::value>(f, dpad, w);
                });
            }
        });
    }
    if (!priv) return;
    __syncthreads();
    // pass 3: add the shared box to the global padded buffer, one atomic per touched site
    for (int i = threadIdx.x; i < vol * M; i += blockDim.x) {
        const float a = sacc[i];
        if (a == 0.0f) continue;
        int r = i, p[S];
        const int k = r / vol;
        r -= k * vol;
        for (int ax = S - 1; ax >= 0; --ax) {
            p[ax] = r % ld[ax] + bmin[ax] - H;
            r /= ld[ax];
        }
        atomicAdd(dpad + ibl::elem_offset(v.L, k, p), a);
    }
}

// ------------------------------------------------------------------------------------ adjoint on spatial bins
//
// The adjoint of random queries sorted by cell (the call runs a counting sort of the query
// indices into spatial bins first, see interp_backward): a bin holds the queries whose coset-0
// cell has padded index P in [b B, (b + 1) B) along every axis (B = 2^LB cells).  Every site such
// a query touches, on any coset, lies in the box [b B - 1 - HALO, (b + 1) B + HALO] per axis (the
// other cosets' cells are the coset-0 cell or the one below it, D <= 2), so a CTA sums a bin's
// contributions in a shared-memory copy of that box and adds the box to the padded gradient
// buffer once, one global atomic per touched site instead of one per (query, site).
// Work items are chunks of at most `chunk` queries of one bin (a bin with many queries is split
// so that clustered queries still spread over the GPU).
// bin of a query for the spatially binned adjoint: the coset-0 cell's padded index per axis
// (the same exact reduction as the kernels), 2^lb cells per bin; -1 for a query that adds
// nothing (non-finite, gout = 0, or its cell outside the padded arrays, so every coset out of
// range)
template <int D>
__device__ __forceinline__ int box_key3(const float (&x)[3], float w, int H2, const ibl::Layout &L, int lb, const int (&nb)[3])
{
    if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2])) || w == 0.0f) return -1;
    int key = 0;
    bool in = true;
    sfor<3>([&](auto A) {
        constexpr int a = decltype(A)::value;
        int i;
        float y;
        reduce_axis<D, 0>(x[a], i, y);
        const int P = i + H2;
        in &= (unsigned)P < (unsigned)L.pdims[a];
        key = key * nb[a] + (P >> lb);
    });
    return in ? key : -1;
}

// bins of 8 cells per axis: boxes of at most 4 x 12^3 (FCC) or 2 x 14^3 (BCC, halo 2) sites, 11 to
// 28 KB, so that four CTAs share an SM (measured on the BCC quintic workload: 16-cell bins, two
// CTAs per SM, 1.33 ms for the box kernel; 8-cell bins, four CTAs, 0.95 ms)
template <class SP>
constexpr int box_lb()
{
    return 3;
}

// resident CTAs per SM of the box kernel (256 threads): as many as the registers allow without
// spilling (4 up to 32 sites; 3 for wider stencils with up to 120 monomials, CC 7-direction: 80
// registers; 2 for CC V_3's 220 monomials)
template <class SP>
constexpr int box_min_blocks()
{
    return SP::NS[0] <= 32 ? 4 : (SP::NMON <= 120 ? 3 : 2);
}

template <class SP, int LB>
constexpr int box_floats()
{
    constexpr int W = (1 << LB) + 2 * SP::HALO + 2;
    return SP::M * W * W * W;
}

struct BoxGrid {
    int nbins;
    int nb[3];      // bins per axis (bin index = (bx nb1 + by) nb2 + bz)
    int chunk;      // queries per work item at most
};

template <class SP, int LB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_adjoint_box(const float4 *__restrict__ rec,
                                                        const int *__restrict__ idx, const int *__restrict__ bin_start,
                                                        const int *__restrict__ item_start, BoxGrid g, DevVol<float> v,
                                                        float *__restrict__ dpad)
{
    static_assert(SP::S == 3 && SP::D <= 2, "3-D lattices with coset spacing 1 or 2");
    constexpr int S = 3, M = SP::M, H = SP::HALO, B = 1 << LB, W = B + 2 * H + 2, VOL = W * W * W;
    extern __shared__ float sacc[];
    const int item = blockIdx.x;
    if (item >= item_start[g.nbins]) return;
    int lo = 0, hi = g.nbins - 1;                         // the item's bin: last b with item_start[b] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    const int bin = lo;
    const int q0 = bin_start[bin] + (item - item_start[bin]) * g.chunk;
    const int q1 = min(q0 + g.chunk, bin_start[bin + 1]);
    int blo[S];
    blo[2] = (bin % g.nb[2]) * B - 1 - H;
    blo[1] = ((bin / g.nb[2]) % g.nb[1]) * B - 1 - H;
    blo[0] = (bin / (g.nb[2] * g.nb[1])) * B - 1 - H;
    constexpr int lstride[S] = {W * W, W, 1};
    for (int i = threadIdx.x; i < M * VOL; i += blockDim.x) sacc[i] = 0.0f;
    __syncthreads();
    // the next query's record (x, y, z, gout: one 16-byte gather) is loaded one iteration ahead
    // (random gathers: their latency hides behind the current query's work)
    float4 nr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (q0 + (int)threadIdx.x < q1) nr = rec[idx[q0 + threadIdx.x]];
    for (int i = q0 + threadIdx.x; i < q1; i += blockDim.x) {
        const float x[S] = {nr.x, nr.y, nr.z};
        const float w = nr.w;
        if (i + (int)blockDim.x < q1) nr = rec[idx[i + blockDim.x]];
        sfor<M>([&](auto Kc) {
            constexpr int K = decltype(Kc)::value;
            const auto f = fold_coset<SP, K, float>(x, v);
            if (!f.in_range) return;
            int lbase = K * VOL, lss[S];
            bool inbox = true;
            sfor<S>([&](auto A) {
                constexpr int a = decltype(A)::value;
                float y;
                int i;
                reduce_axis<SP::D, SP::COSET[K][a]>(x[a], i, y);
                const int lp = i + 2 * H - blo[a];        // box coordinate of the cell's site
                inbox &= lp >= H && lp < W - H;            // its stencil inside the box
                lbase += lp * lstride[a];
                int st = lstride[0];
                sfor<S - 1>([&](auto Bc) {
                    if (f.sl[A].ax == 1 + decltype(Bc)::value) st = lstride[1 + decltype(Bc)::value];
                });
                lss[A] = f.sl[A].sg * st;
            });
            // always inside for a query of this bin (the binning takes the same cell); a query
            // outside would add straight to the global buffer
            sfor<SP::K>([&](auto Jc) {
                if (f.piece == decltype(Jc)::value) {
                    if (inbox) adjoint_piece_local<SP, decltype(Jc)::value>(f, lss, lbase, sacc, w);
                    else adjoint_piece<SP, decltype(Jc)::value>(f, dpad, w);
                }
            });
        });
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M * VOL; i += blockDim.x) {
        const float a = sacc[i];
        if (a == 0.0f) continue;
        const int k = i / VOL;
        const int r = i - k * VOL;
        const int p[S] = {blo[0] + r / (W * W), blo[1] + (r / W) % W, blo[2] + r % W};
        bool in = true;
        int off = k * v.L.kw;
        sfor<S>([&](auto A) {
            constexpr int LB = axis_lb<SP, float>(decltype(A)::value);
            in &= (unsigned)p[A] < (unsigned)v.L.pdims[A];
            off += (p[A] >> LB) * v.L.bstride[A] + (p[A] & ((1 << LB) - 1)) * v.L.wt[A];
        });
        if (in) atomicAdd(dpad + off, a);
    }
}

}  // namespace ib
