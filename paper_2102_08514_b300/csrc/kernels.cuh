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
//   3. branch-free sub-region index: q = sum_i [p_i . y' - d_i >= 0] 2^i, j = sigma[q mod r]
//      (Sec. 4.2; sigma is packed into one 64-bit constant);
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

// coset shifts packed 4 bits per coordinate, so a run-time coset index can read them
template <class SP>
constexpr uint64_t cosets_packed()
{
    uint64_t v = 0;
    for (int k = 0; k < SP::M; ++k)
        for (int a = 0; a < SP::S; ++a) v |= (uint64_t)SP::COSET[k][a] << (4 * (k * SP::S + a));
    return v;
}

// one slot of the folded offset: |y| and what the gather needs about the original axis it came
// from (sign, within-brick coordinate of the cell, brick geometry of that axis)
struct Slot {
    float y;
    int sg;   // +1 / -1: sign of y along the original axis
    int ax;   // original axis
    int p;    // within-brick coordinate of the cell's padded index along that axis
    int lb;   // log2 brick width of that axis
    int bs;   // brick stride of that axis
    int wt;   // within-brick weight of that axis
};

__device__ __forceinline__ void cswap(Slot &a, Slot &b)
{
    // descending order; ties keep the current order (either order is valid on a chamber wall)
    const bool sw = a.y < b.y;
    const Slot lo = sw ? a : b;
    const Slot hi = sw ? b : a;
    a = hi;
    b = lo;
}

template <int S>
__device__ __forceinline__ void sort_desc(Slot (&sl)[S])
{
    if constexpr (S == 2) {
        cswap(sl[0], sl[1]);
    } else if constexpr (S == 3) {
        cswap(sl[0], sl[1]); cswap(sl[1], sl[2]); cswap(sl[0], sl[1]);
    } else if constexpr (S == 4) {
        cswap(sl[0], sl[1]); cswap(sl[2], sl[3]); cswap(sl[0], sl[2]); cswap(sl[1], sl[3]); cswap(sl[1], sl[2]);
    }
}

template <class SP>
constexpr uint64_t sigma_packed()
{
    uint64_t v = 0;
    for (int r = 0; r < SP::R; ++r) v |= (uint64_t)(SP::SIGMA[r] < 0 ? 15 : SP::SIGMA[r]) << (4 * r);
    return v;
}

// ------------------------------------------------------------------------------------ volume

template <class CT> struct DevVol {
    const CT *c;        // padded, bricked coset arrays, coset-major
    ibl::Layout L;
};

template <int S> struct Fold {
    int base;           // element offset of the brick holding the cell's site (coset included)
    float t[S];         // folded offset y' (before the anchor shift)
    Slot sl[S];         // per folded slot: sign, original axis and brick geometry
    int piece;
    bool in_range;
};

// element offset, relative to Fold::base, of the site displaced by o along folded slot A
__device__ __forceinline__ int slot_term(const Slot &sl, int o)
{
    const int v = sl.p + sl.sg * o;
    return (v >> sl.lb) * sl.bs + (v & ((1 << sl.lb) - 1)) * sl.wt;
}

// steps 1-3 for coset K of spline SP (K < 0: the run-time coset index kr)
template <class SP, int K, class CT>
__device__ __forceinline__ Fold<SP::S> fold_coset(const float (&x)[SP::S], const DevVol<CT> &v, int kr = 0)
{
    constexpr int S = SP::S;
    constexpr int H = SP::HALO;
    constexpr int ESZ = (int)sizeof(CT);
    Fold<S> f;
    bool ok = true;
    int base = (K >= 0 ? K : kr) * v.L.coset_elems;
    sfor<S>([&](auto A) {
        constexpr int a = decltype(A)::value;
        constexpr int lb = ibl::brick_lb(S, ESZ, a);
        int idx;
        float y;
        if constexpr (K >= 0) {
            reduce_axis<SP::D, SP::COSET[K][a]>(x[a], idx, y);
        } else {
            constexpr uint64_t packed = cosets_packed<SP>();
            const int l = (int)((packed >> (4 * (kr * S + a))) & 15u);
            reduce_axis_rt<SP::D>(x[a], l, idx, y);
        }
        ok &= (unsigned)(idx + H) < (unsigned)(v.L.n[a] + 2 * H);
        const int P = idx + 2 * H;                       // padded index of the cell's site
        base += (P >> lb) * v.L.bstride[a];
        Slot &sl = f.sl[a];
        sl.y = fabsf(y);
        sl.sg = (y < 0.0f) ? -1 : 1;
        sl.ax = a;
        sl.p = P & ((1 << lb) - 1);
        sl.lb = lb;
        sl.bs = v.L.bstride[a];
        sl.wt = v.L.wt[a];
    });
    sort_desc<S>(f.sl);
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
            q |= (acc >= 0.0f ? 1u : 0u) << i;
        });
        constexpr uint64_t packed = sigma_packed<SP>();
        j = (int)((packed >> (4 * (q % (unsigned)SP::R))) & 15u);
    }
    f.piece = j;
    f.base = base;
    f.in_range = ok;
    return f;
}

// element offset (relative to Fold::base) of stencil site M of piece J
template <class SP, int J, int M>
__device__ __forceinline__ int site_offset(const Fold<SP::S> &f)
{
    int off = 0;
    sfor<SP::S>([&](auto A) {
        constexpr int g = SP::SITE[J][M][decltype(A)::value];
        off += slot_term(f.sl[A], g);
    });
    return off;
}

// steps 4-5 for piece J: accumulate f (and grad f if GRAD) into the query's sums
template <class SP, int J, bool GRAD, class CT>
__device__ __forceinline__ void eval_piece(const Fold<SP::S> &f, const DevVol<CT> &v, float &val, float (&grad)[SP::S])
{
    constexpr int S = SP::S;
    constexpr int NS = SP::NS[J];
    constexpr int NM = SP::NMON;
    const CT *cb = v.c + f.base;
    float c[NS];
    sfor<NS>([&](auto Mi) { c[Mi] = load_coef<CT>(cb + site_offset<SP, J, decltype(Mi)::value>(f)); });
    float t[S];
    sfor<S>([&](auto A) {
        constexpr float an = SP::ANCHOR[J][decltype(A)::value];
        t[A] = f.t[A] - an;
    });
    float b[NM];
    sfor<NM>([&](auto A) { b[A] = 0.0f; });
    accumulate<NS, NM>(b, c, typename SP::template NZL<J>{});
    if constexpr (!GRAD) {
        val += horner<S, S, SP::DEG, 0, NM>(b, t);
    } else {
        VG<S> r = horner_grad<S, S, SP::DEG, 0, NM>(b, t);
        val += r.v;
        // back through the fold: d/dx_ax = sign * d/dy'_slot
        sfor<S>([&](auto A) {
            const float gs = (f.sl[A].sg < 0) ? -r.g[A] : r.g[A];
            sfor<S>([&](auto B) { grad[B] += (f.sl[A].ax == B) ? gs : 0.0f; });
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
    } else {
        // several pieces: one copy of each piece's code, run-time coset loop
#pragma unroll 1
        for (int k = 0; k < SP::M; ++k) {
            const auto f = fold_coset<SP, -1, CT>(x, v, k);
            if (f.in_range) {
                sfor<SP::K>([&](auto Jc) {
                    if (f.piece == decltype(Jc)::value) eval_piece<SP, decltype(Jc)::value, GRAD, CT>(f, v, val, grad);
                });
            }
        }
    }
}

// MODE 0: out = f.  MODE 1: out = f (if out), grad = grad f.  MODE 2: grad = gout * grad f.
template <class SP, class CT, int MODE>
__global__ void __launch_bounds__(128) k_eval(const float *__restrict__ pts, int64_t n, DevVol<CT> v,
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
