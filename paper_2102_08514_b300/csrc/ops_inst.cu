// ops_inst.cu -- instantiates the kernels of ONE spline and ONE kernel family.  The build
// compiles this file once per (spline, family) with -DINTERP_SPLINE=<name> -DINTERP_PART=<0..3>
// so the large unrolled kernels compile in parallel.
#include <algorithm>
#include <atomic>

#include "kernels.cuh"
#include "registry.h"

#ifndef INTERP_SPLINE
#error "compile with -DINTERP_SPLINE=<spline struct name>"
#endif
#ifndef INTERP_PART
#error "compile with -DINTERP_PART=<0..3>"
#endif

#define IB_CAT2(a, b, c, d) a##b##c##d
#define IB_CAT(a, b, c, d) IB_CAT2(a, b, c, d)

namespace {

constexpr int kTPB = 128;
using SP = interp_gen::INTERP_SPLINE;

template <class CT>
ib::DevVol<CT> make_vol(const void *c, const ibl::Layout &L)
{
    ib::DevVol<CT> v;
    v.c = static_cast<const CT *>(c);
    v.L = L;
    return v;
}

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kTPB - 1) / kTPB); }

// shared memory a CTA may use (opt-in maximum on sm_100 / sm_103)
constexpr size_t kMaxSmem = 227 * 1024;

constexpr int nnz_sum()
{
    int t = 0;
    for (int j = 0; j < SP::K; ++j) t += SP::NNZ[j];
    return t;
}

// CTA residency the plain evaluation kernel's registers are fitted to.  One-piece splines with
// wide stencils and the one-pass accumulation of b (>= 48 sites, <= 120 monomials: CC
// 7-direction) get up to 128 registers (4 CTAs per SM): a query's gathers issue closer together
// and its sectors are reused in L1 before they are evicted (measured, CC 7-direction on 256^3,
// 2^24 random queries: 26.3 -> 18.7 L1 misses per query for its 15.0 distinct sectors, value
// 1.563 -> 1.278 ms; spatially sorted queries 0.64 -> 0.70 ms).  The others are unbounded (the
// compiler's choice, 55-72 registers; CC V_3's blocked accumulation measured no faster).
constexpr int eval_min_blocks()
{
    return (SP::K == 1 && SP::NSMAX >= 48 && SP::NMON <= 120) ? 4 : 1;
}

// whether the plain evaluation runs the warp-cooperative gathers (k_eval_coop): one-piece
// splines with 24 to 32 stencil sites per query (all cosets), whose sites fill most of one load
// instruction of a warp.  Measured, 2^24 random queries: BCC quintic (32 sites) value 0.822 ->
// 0.673 ms, value + grad 0.878 -> 0.780 ms (L1 -> L2 requests 13.0 -> 9.1 per query); CC
// 7-direction (53 sites, two rounds per query) value 1.278 -> 1.337 ms (the table's shared-
// memory traffic outweighs the fewer requests), so longer stencils keep k_eval.
constexpr bool coop_eval()
{
    return SP::K == 1 && SP::M * SP::NS[0] >= 24 && SP::M * SP::NS[0] <= 32;
}

// resident CTAs per SM the cooperative kernel's registers are fitted to: 8 for values (64
// registers), 6 with the gradient (80 registers; at 64 it spills)
template <int MODE>
constexpr int coop_min_blocks()
{
    return MODE == 0 ? 8 : 6;
}

// whether the piece-binned kernels are the default for evaluation (GRAD: value + gradient).
// Sorting a tile's items by piece pays when the pieces' divergent work is large: the plain kernel
// shares all but the accumulation of b between the pieces, so a warp pays the sum of the pieces'
// nonzeros once per coset.  Measured, 2^24 / 2^22 random queries, plain against binned: FCC V_1
// (4 pieces, 74 nonzeros in all) value 0.175 / 0.323 ms, value + grad 0.208 / 0.358 ms; BCC V_1
// (14 pieces, 848) 0.900 / 0.649, 0.960 / 0.787; FCC V_2 (4, 1361) 0.774 / 0.554; D4* (6, 5530)
// 6.76 / 2.82 ms.  Rays (RAYS) of value + gradient with small pieces stay plain (BCC V_1,
// 1024^2 x 256: value 11.66 / 11.23 ms, value + grad 12.32 / 15.69 ms).
template <bool GRAD, bool RAYS>
constexpr bool binned_default()
{
    if constexpr (SP::K < 4 || nnz_sum() < 200) return false;
    else return !(RAYS && GRAD && SP::NNZMAX <= 100);
}

// a kernel attribute is set once per device: one bit per device (devices >= 64 set it every call);
// several host threads may launch at once
inline bool attr_pending(const std::atomic<unsigned long long> &done, int dev)
{
    return dev >= 64 || !((done.load(std::memory_order_acquire) >> dev) & 1ull);
}
inline void attr_set(std::atomic<unsigned long long> &done, int dev)
{
    if (dev < 64) done.fetch_or(1ull << dev, std::memory_order_release);
}

// piece-binned kernel configurations: (tile of queries, threads per CTA)
template <class CT, int MODE, int T, int NT, bool DENSE = false>
[[maybe_unused]] cudaError_t launch_binned_cfg(const float *pts, int64_t n, const void *c, const ibl::Layout &L,
                                               float *out, float *grad, const float *gout, cudaStream_t st)
{
    constexpr size_t smem = ib::binned_smem_bytes<SP, MODE, T>();
    static_assert(smem <= kMaxSmem, "binned tile must fit shared memory");
    auto kern = ib::k_eval_binned<SP, CT, MODE, T, NT, DENSE>;
    static std::atomic<unsigned long long> configured{0};   // per device: the attribute is set once
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_pending(configured, dev)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set(configured, dev);
    }
    const unsigned grid = (unsigned)((n + T - 1) / T);
    kern<<<grid, NT, smem, st>>>(pts, n, make_vol<CT>(c, L), out, grad, gout);
    return cudaPeekAtLastError();
}

// queries per tile of the piece-binned kernels.  Each tile re-fetches the code of every piece it
// meets, so splines with large pieces (>= 400 nonzeros, instruction-fetch bound) take 2048-query
// tiles; the others 1024.  The tile's shared memory stays within 170 KB: beyond that the L1 data
// cache left for the coefficient gathers is too small (measured: BCC V_2 value+grad 12.2 -> 6.8 ms
// with 2048-query tiles (168 KB); BCC V_1 (75 nonzeros) 0.82 -> 1.01 ms; D4* value+grad
// 4.2 -> 7.1 ms at 200 KB).  8-coset D4 drops to 512 / 256.
constexpr size_t kBinSmemBudget = 170 * 1024;

template <int MODE>
constexpr int bin_tile()
{
    if constexpr (SP::NNZMAX >= 400 && ib::binned_smem_bytes<SP, MODE, 2048>() <= kBinSmemBudget &&
                  SP::M * 2048 <= 65535)
        return 2048;
    else
        return ib::binned_smem_bytes<SP, MODE, 1024>() <= kBinSmemBudget ? 1024
               : ib::binned_smem_bytes<SP, MODE, 512>() <= kBinSmemBudget ? 512 : 256;
}

template <class CT, int MODE>
[[maybe_unused]] cudaError_t launch_eval_binned(const float *pts, int64_t n, const void *c, const ibl::Layout &L,
                                                float *out, float *grad, const float *gout, int flags, cudaStream_t st)
{
    if constexpr (SP::K > 1) {
        // FLAG_BIN_SMALL: 256-query tiles on 128-thread CTAs (several CTAs per SM)
        if (flags & ibr::FLAG_BIN_SMALL) return launch_binned_cfg<CT, MODE, 256, 128>(pts, n, c, L, out, grad, gout, st);
        if constexpr (SP::DENSE) {
            // the dense piece tables (one shared code path for all pieces) are slower here than the
            // unrolled per-piece code, whose 1.8x fewer FMAs outweigh its instruction fetch
            // (measured, BCC V_2, 2^24 random queries: value 5.65 vs 8.67 ms, value+grad 6.81 vs
            // 9.99 ms); FLAG_DENSE_ON selects them
            if (flags & ibr::FLAG_DENSE_ON)
                return launch_binned_cfg<CT, MODE, bin_tile<MODE>(), 512, true>(pts, n, c, L, out, grad, gout, st);
        }
        return launch_binned_cfg<CT, MODE, bin_tile<MODE>(), 512>(pts, n, c, L, out, grad, gout, st);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <class CT, int MODE>
cudaError_t launch_eval(const float *pts, int64_t n, const void *c, const ibl::Layout &L, float *out, float *grad,
                        const float *gout, int, cudaStream_t st)
{
    if constexpr (coop_eval())
        ib::k_eval_coop<SP, CT, MODE, coop_min_blocks<MODE>()><<<grid_for(n), kTPB, 0, st>>>(pts, n, make_vol<CT>(c, L),
                                                                                               out, grad, gout);
    else
        ib::k_eval<SP, CT, MODE, eval_min_blocks()><<<grid_for(n), kTPB, 0, st>>>(pts, n, make_vol<CT>(c, L), out,
                                                                                   grad, gout);
    return cudaPeekAtLastError();
}

[[maybe_unused]] cudaError_t launch_adjoint(const float *pts, int64_t n, const float *gout, const ibl::Layout &L,
                                            float *dpad, cudaStream_t st)
{
    if constexpr (SP::S == 3 && SP::K < 4) {
        // blocks of sorted queries fit a shared-memory box: privatised sums (3-D)
        const unsigned grid = (unsigned)((n + ib::kAdjChunk - 1) / ib::kAdjChunk);
        ib::k_adjoint_priv<SP><<<grid, 256, 0, st>>>(pts, n, gout, make_vol<float>(nullptr, L), dpad);
    } else if constexpr (SP::K >= 4) {
        // many pieces: sort each tile's items by piece first, then scatter with global atomics
        // (divergence over the pieces costs more than the privatised box saves)
        constexpr int T = ib::binned_adjoint_smem_bytes<SP, 1024>() <= kMaxSmem ? 1024
                          : ib::binned_adjoint_smem_bytes<SP, 512>() <= kMaxSmem ? 512 : 256;
        constexpr int NT = 512;
        constexpr size_t smem = ib::binned_adjoint_smem_bytes<SP, T>();
        static_assert(smem <= kMaxSmem, "binned adjoint tile must fit shared memory");
        auto kern = ib::k_adjoint_binned<SP, T, NT>;
        static std::atomic<unsigned long long> configured{0};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (attr_pending(configured, dev)) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set(configured, dev);
        }
        kern<<<(unsigned)((n + T - 1) / T), NT, smem, st>>>(pts, n, gout, make_vol<float>(nullptr, L), dpad);
    } else {
        // a 4-D box with its stencil halo does not fit shared memory: direct atomics
        ib::k_adjoint<SP><<<grid_for(n), kTPB, 0, st>>>(pts, n, gout, make_vol<float>(nullptr, L), dpad);
    }
    return cudaPeekAtLastError();
}

template <int LB, int MINB>
[[maybe_unused]] cudaError_t launch_adjoint_box_cfg(const ibr::BoxArgs &a, const ibl::Layout &L, float *dpad,
                                                    cudaStream_t st)
{
    constexpr size_t smem = (size_t)ib::box_floats<SP, LB>() * sizeof(float);
    static_assert(smem <= kMaxSmem, "adjoint box must fit shared memory");
    auto kern = ib::k_adjoint_box<SP, LB, MINB>;
    static std::atomic<unsigned long long> configured{0};   // per device: the attribute is set once
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_pending(configured, dev)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set(configured, dev);
    }
    ib::BoxGrid g;
    g.nbins = a.nbins;
    g.nb[0] = a.nb[0];
    g.nb[1] = a.nb[1];
    g.nb[2] = a.nb[2];
    g.chunk = a.chunk;
    kern<<<(unsigned)a.max_items, 256, smem, st>>>(reinterpret_cast<const float4 *>(a.rec), a.idx, a.bin_start,
                                                    a.item_start, g, make_vol<float>(nullptr, L), dpad);
    return cudaPeekAtLastError();
}

[[maybe_unused]] cudaError_t launch_adjoint_box(const ibr::BoxArgs &a, const ibl::Layout &L, float *dpad, cudaStream_t st)
{
    if constexpr (SP::S == 3 && SP::K < 4 && SP::D <= 2) {
        constexpr int LB = ib::box_lb<SP>();
        if (a.lb != LB) return cudaErrorInvalidValue;
        return launch_adjoint_box_cfg<LB, ib::box_min_blocks<SP>()>(a, L, dpad, st);
    } else {
        return cudaErrorInvalidValue;
    }
}

// counting sort of the queries by Morton-ordered bins: count, exclusive scan, scatter
[[maybe_unused]] cudaError_t launch_sort(const float *pts, int64_t n, const ibl::Layout &L, int bb, int bits,
                                         unsigned *keys, int nkeys, int32_t *perm, float *pts_out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(keys, 0, (size_t)nkeys * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaGetLastError();
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16);
    ib::k_sort_count<SP><<<grid, 256, 0, st>>>(pts, n, L, bb, bits, keys);
    // exclusive scan of the counters; the block sums live right after them
    const int nblk = (nkeys + ib::kScanBlock - 1) / ib::kScanBlock;
    unsigned *sums = keys + nkeys;
    ib::k_scan_block_sums<1024><<<nblk, 1024, 0, st>>>(keys, nkeys, sums);
    ib::k_scan_exclusive<1024><<<1, 1024, 0, st>>>(sums, nblk);
    ib::k_scan_apply<1024><<<nblk, 1024, 0, st>>>(keys, nkeys, sums);
    ib::k_sort_scatter<SP><<<grid, 256, 0, st>>>(pts, n, L, bb, bits, keys, perm, pts_out);
    return cudaPeekAtLastError();
}

[[maybe_unused]] cudaError_t launch_debug(const float *pts, int64_t n, const ibl::Layout &L, int32_t *cells,
                                          int32_t *piece, cudaStream_t st)
{
    ib::k_debug<SP><<<grid_for(n), kTPB, 0, st>>>(pts, n, make_vol<float>(nullptr, L), cells, piece);
    return cudaPeekAtLastError();
}

template <bool GRAD>
[[maybe_unused]] cudaError_t launch_rays(const ibl::RayGeom &rg, const void *c, const ibl::Layout &L, float *out,
                                         float *pts_out, int flags, cudaStream_t st)
{
    if constexpr (SP::S == 3) {
        if constexpr (SP::K > 1) {
            // multi-piece splines: whole rays per tile, samples binned by piece (default as
            // binned_default, FLAG_BINNED_OFF / FLAG_BINNED_ON force the plain / binned kernel)
            constexpr int T = bin_tile<GRAD ? 1 : 0>();
            const bool want = (flags & ibr::FLAG_BINNED_ON)    ? true
                              : (flags & ibr::FLAG_BINNED_OFF) ? false
                                                               : binned_default<GRAD, true>();
            if (want && rg.steps >= 1 && rg.steps <= T) {
                constexpr size_t smem = ib::binned_smem_bytes<SP, GRAD ? 1 : 0, T>();
                static_assert(smem <= kMaxSmem, "binned tile must fit shared memory");
                // rays of a dense-table spline use the tables (measured, BCC V_2, 1024^2 x 256: value
                // 127 -> 104 ms, value+grad 151 -> 104 ms); FLAG_DENSE_OFF selects the unrolled code
                const bool dense = SP::DENSE && !(flags & ibr::FLAG_DENSE_OFF);
                auto kd = ib::k_rays_binned<SP, GRAD, T, 512, SP::DENSE>;
                auto kp = ib::k_rays_binned<SP, GRAD, T, 512>;
                auto kern = dense ? kd : kp;
                static std::atomic<unsigned long long> configured{0};   // both variants, once per device
                int dev = 0;
                cudaError_t e = cudaGetDevice(&dev);
                if (e != cudaSuccess) return e;
                if (attr_pending(configured, dev)) {
                    e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (e == cudaSuccess && SP::DENSE)
                        e = cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (e != cudaSuccess) return e;
                    attr_set(configured, dev);
                }
                const int64_t rays = (int64_t)rg.width * rg.height;
                const int rt = T / rg.steps;
                kern<<<(unsigned)((rays + rt - 1) / rt), 512, smem, st>>>(rg, make_vol<float>(c, L), out, pts_out);
                return cudaPeekAtLastError();
            }
        }
        const dim3 grid((rg.width + 15) / 16, (rg.height + 7) / 8);
        ib::k_rays<SP, GRAD><<<grid, 128, 0, st>>>(rg, make_vol<float>(c, L), out, pts_out);
        return cudaPeekAtLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

}  // namespace

namespace ibr {

void IB_CAT(fill_, INTERP_SPLINE, _, INTERP_PART)(SplineOps &o)
{
#if INTERP_PART == 3
    o.name = SP::NAME;
    o.s = SP::S;
    o.nxi = SP::NXI;
    o.kind = SP::KIND;
    o.M = SP::M;
    o.D = SP::D;
    o.detl = SP::DETL;
    o.halo = SP::HALO;
    o.K = SP::K;
    o.deg = SP::DEG;
    o.nmon = SP::NMON;
    o.xi = &SP::XI[0][0];
    o.cosets = &SP::COSET[0][0];
    o.fma_value = SP::FMA_VALUE;
    o.fma_grad = SP::FMA_GRAD;
    o.lookups = SP::LOOKUPS;
    o.nnz_sum = nnz_sum();
    o.binned_eval = binned_default<false, false>();
    o.coop_eval = coop_eval();
    o.adjoint = launch_adjoint;
    if constexpr (SP::S == 3 && SP::K < 4 && SP::D <= 2) {
        o.adjoint_box = launch_adjoint_box;
        o.box_lb = ib::box_lb<SP>();
    }
    o.debug = launch_debug;
    o.sort = launch_sort;
    if constexpr (SP::S == 3) {
        o.rays[0] = launch_rays<false>;
        o.rays[1] = launch_rays<true>;
    }
#else
    constexpr int mode = INTERP_PART;
    o.eval[0][mode] = launch_eval<float, mode>;
    if constexpr (SP::HALF_STORAGE) {
        o.eval[1][mode] = launch_eval<__half, mode>;
        o.eval[2][mode] = launch_eval<__nv_bfloat16, mode>;
    }
    if constexpr (SP::K > 1) {
        o.eval_binned[0][mode] = launch_eval_binned<float, mode>;
        if constexpr (SP::HALF_STORAGE) {
            o.eval_binned[1][mode] = launch_eval_binned<__half, mode>;
            o.eval_binned[2][mode] = launch_eval_binned<__nv_bfloat16, mode>;
        }
    }
#endif
}

}  // namespace ibr
