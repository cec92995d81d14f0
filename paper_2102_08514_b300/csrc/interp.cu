// interp.cu -- C ABI of the lattice convolution-sum evaluator (see include/interp.h).
//
// Host side: handle creation (matching (L, Xi) against the generated splines), halo-padded
// coefficient storage, conversion of user coefficients, and launches of the kernels in
// kernels.cuh on the caller's stream.  No host computation of results, no fallback path.
#include "interp.h"

#include <algorithm>
#include <atomic>
#include <array>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <type_traits>

#include "generated/splines.h"

#include "kernels.cuh"
#include "registry.h"

INTERP_GEN_SPLINES(INTERP_FILL_DECL)

namespace {

using ibr::SplineOps;
constexpr int kTPB = 128;

#define INTERP_OPS_ENTRY(name)           \
    [] {                                 \
        SplineOps o;                     \
        ibr::fill_##name##_0(o);         \
        ibr::fill_##name##_1(o);         \
        ibr::fill_##name##_2(o);         \
        ibr::fill_##name##_3(o);         \
        return o;                        \
    }(),
const std::vector<SplineOps> &registry()
{
    static const std::vector<SplineOps> r = {INTERP_GEN_SPLINES(INTERP_OPS_ENTRY)};
    return r;
}
#undef INTERP_OPS_ENTRY

// ------------------------------------------------------------------------------------ conversion kernels

template <class ST, class CT>
__device__ __forceinline__ CT convert_to(ST x)
{
    if constexpr (std::is_same_v<ST, double>) {
        // round once, directly from FP64 to the storage type
        if constexpr (std::is_same_v<CT, float>) return (float)x;
        else if constexpr (std::is_same_v<CT, __half>) return __double2half(x);
        else return __double2bfloat16(x);
    } else {
        float f;
        if constexpr (std::is_same_v<ST, __half>) f = __half2float(x);
        else if constexpr (std::is_same_v<ST, __nv_bfloat16>) f = __bfloat162float(x);
        else f = x;
        if constexpr (std::is_same_v<CT, float>) return f;
        else if constexpr (std::is_same_v<CT, __half>) return __float2half_rn(f);
        else return __float2bfloat16_rn(f);
    }
}

// padded, bricked element offset of unpadded linear element e (coset-major, row-major)
__device__ __forceinline__ int padded_offset(const ibl::Layout &L, int64_t e)
{
    int p[4] = {0, 0, 0, 0};
    for (int a = L.s - 1; a >= 0; --a) {
        p[a] = (int)(e % L.n[a]) + L.pad;
        e /= L.n[a];
    }
    return ibl::elem_offset(L, (int)e, p);
}

// copy src (unpadded, coset-major, row-major) into the interior of the padded, bricked arrays
template <class ST, class CT>
__global__ void k_pad_copy(const ST *__restrict__ src, CT *__restrict__ dst, int64_t total, ibl::Layout L)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        dst[padded_offset(L, e)] = convert_to<ST, CT>(src[e]);
}

// the taps of a lattice filter resolved per output coset: tap t of output coset k reads the
// samples of coset src[k][t] at index i + shift[k][t], i.e. at linear offset delta[k][t] from
// the output's own sample (passed by value as a kernel parameter)
constexpr int kMaxTaps = 64;
struct PrefilterTaps {
    int ntaps;
    int reach;                       // largest |shift| over taps and axes
    float w[kMaxTaps];
    int delta[8][kMaxTaps];
    unsigned char neg[8][kMaxTaps];  // axes on which the tap's index shift is -1 (reach 1)
    unsigned char pos[8][kMaxTaps];  // axes on which it is +1
    signed char src[8][kMaxTaps];
    signed char shift[8][kMaxTaps][4];
};

// c_k[i] = sum_t w_t f_src[i + shift] over the taps (samples taken as zero outside the arrays),
// rounded to the storage type and written to the interior of the padded, bricked arrays.
// A thread computes the outputs of all M cosets at PF_RUN consecutive sites along the last axis,
// so the taps of every coset read the same neighbourhood of every coset array while it is in
// cache (each input is fetched from DRAM about once) and each tap's address and bounds test serve
// PF_RUN loads.  A CTA covers whole rows (all axes but the last fixed).  Bounds are tested without
// branches (face masks against the taps' sign masks) for filters that reach one index step (all
// filters on nearest neighbours), per tap and axis for longer ones.
constexpr int PF_RUN = 4;

template <class CT>
__global__ void __launch_bounds__(256) k_prefilter(const float *__restrict__ f, CT *__restrict__ dst, ibl::Layout L,
                                                   int lw, int chunks, int nrows, int M, int cstride, PrefilterTaps tp)
{
    const int s = L.s, nl = L.n[s - 1];
    int row, i0;                                     // the thread's first site on the row
    if (chunks == 1) {                               // several rows of 2^lw threads per CTA
        row = blockIdx.x * (blockDim.x >> lw) + (threadIdx.x >> lw);
        i0 = (threadIdx.x & ((1 << lw) - 1)) * PF_RUN;
    } else {                                         // rows longer than a CTA: `chunks` CTAs per row
        row = blockIdx.x / chunks;
        i0 = ((blockIdx.x % chunks) * blockDim.x + threadIdx.x) * PF_RUN;
    }
    if (row >= nrows || i0 >= nl) return;
    int idx[4] = {0, 0, 0, 0};
    int r = row;
    for (int a = s - 2; a >= 0; --a) {
        idx[a] = r % L.n[a];
        r /= L.n[a];
    }
    const int la = s - 1;
    const int e0 = row * nl + i0;                    // linear index of the first site within a coset
    int p[4];
    for (int a = 0; a < 4; ++a) p[a] = idx[a] + L.pad;
    if (tp.reach <= 1) {
        // face masks of the axes but the last (shared by the run) and per site of the last axis
        unsigned lo = 0, hi = 0;
        for (int a = 0; a < la; ++a) {
            lo |= (idx[a] == 0 ? 1u : 0u) << a;
            hi |= (idx[a] == L.n[a] - 1 ? 1u : 0u) << a;
        }
        unsigned lo_u[PF_RUN], hi_u[PF_RUN];
        bool live[PF_RUN];
#pragma unroll
        for (int u = 0; u < PF_RUN; ++u) {
            const int il = i0 + u;
            live[u] = il < nl;
            lo_u[u] = lo | ((il == 0 ? 1u : 0u) << la);
            hi_u[u] = hi | ((il == nl - 1 ? 1u : 0u) << la);
        }
#pragma unroll 1
        for (int k = 0; k < M; ++k) {
            const float *fk = f + k * cstride + e0;
            float acc[PF_RUN];
#pragma unroll
            for (int u = 0; u < PF_RUN; ++u) acc[u] = 0.0f;
#pragma unroll 2
            for (int t = 0; t < tp.ntaps; ++t) {
                const unsigned ng = tp.neg[k][t], ps = tp.pos[k][t];
                const int d = tp.delta[k][t];
                const float w = tp.w[t];
                float v[PF_RUN];
#pragma unroll
                for (int u = 0; u < PF_RUN; ++u) {
                    // a tap outside the arrays (or a site past the row) reads the run's first
                    // sample, always in bounds, and contributes 0
                    const bool in = live[u] && !((ng & lo_u[u]) | (ps & hi_u[u]));
                    const float x = __ldg(fk + (in ? d + u : 0));
                    v[u] = in ? x : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < PF_RUN; ++u) acc[u] = fmaf(w, v[u], acc[u]);
            }
#pragma unroll
            for (int u = 0; u < PF_RUN; ++u) {
                if (!live[u]) break;
                p[la] = i0 + u + L.pad;
                dst[ibl::elem_offset(L, k, p)] = convert_to<float, CT>(acc[u]);
            }
        }
        return;
    }
    // longer filters: explicit bounds per tap and axis
    for (int u = 0; u < PF_RUN && i0 + u < nl; ++u) {
        idx[la] = i0 + u;
        p[la] = idx[la] + L.pad;
#pragma unroll 1
        for (int k = 0; k < M; ++k) {
            const int e = k * cstride + e0 + u;
            float acc = 0.0f;
            for (int t = 0; t < tp.ntaps; ++t) {
                bool in = true;
                for (int a = 0; a < s; ++a) {
                    const int j = idx[a] + tp.shift[k][t][a];
                    in &= (unsigned)j < (unsigned)L.n[a];
                }
                if (in) acc = fmaf(tp.w[t], __ldg(f + e + tp.delta[k][t]), acc);
            }
            dst[ibl::elem_offset(L, k, p)] = convert_to<float, CT>(acc);
        }
    }
}

// dst (unpadded FP32) += interior of the padded FP32 gradient buffer
__global__ void k_unpad_add(const float *__restrict__ pad_buf, float *__restrict__ dst, int64_t total, ibl::Layout L)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] += pad_buf[padded_offset(L, e)];
}

// ------------------------------------------------------------------------------------ exact integer helpers

int64_t idet(const int64_t *a, int m)
{
    if (m == 1) return a[0];
    int64_t sum = 0, sub[16];
    for (int c = 0; c < m; ++c) {
        int k = 0;
        for (int r = 1; r < m; ++r)
            for (int cc = 0; cc < m; ++cc)
                if (cc != c) sub[k++] = a[r * m + cc];
        sum += ((c & 1) ? -1 : 1) * a[c] * idet(sub, m - 1);
    }
    return sum;
}

// adj such that adj * L = det * I
void iadj(const int64_t *B, int m, int64_t *adj)
{
    if (m == 1) {
        adj[0] = 1;
        return;
    }
    int64_t sub[16];
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) {
            int k = 0;
            for (int r = 0; r < m; ++r) {
                if (r == a) continue;
                for (int cc = 0; cc < m; ++cc)
                    if (cc != c) sub[k++] = B[r * m + cc];
            }
            adj[c * m + a] = (((a + c) & 1) ? -1 : 1) * idet(sub, m - 1);
        }
}

struct LatticeInfo {
    int D = 0;
    std::vector<std::array<int, 4>> cosets;
};

// D (smallest with D Z^s inside L Z^s) and the coset shifts in [0, D)^s
bool lattice_info(int s, const int32_t *L, LatticeInfo &li)
{
    int64_t B[16], A[16];
    for (int k = 0; k < s * s; ++k) B[k] = L[k];
    const int64_t det = idet(B, s);
    if (det == 0) return false;
    iadj(B, s, A);
    const int64_t ad = det < 0 ? -det : det;
    auto member = [&](const int *z) {
        for (int r = 0; r < s; ++r) {
            int64_t acc = 0;
            for (int c = 0; c < s; ++c) acc += A[r * s + c] * z[c];
            if (acc % ad != 0) return false;
        }
        return true;
    };
    for (int d = 1; d <= ad; ++d) {
        bool all = true;
        for (int a = 0; a < s && all; ++a) {
            int z[4] = {0, 0, 0, 0};
            z[a] = d;
            all = member(z);
        }
        if (all) {
            li.D = d;
            break;
        }
    }
    if (li.D == 0 || li.D > 16) return false;
    int total = 1;
    for (int a = 0; a < s; ++a) total *= li.D;
    for (int e = 0; e < total; ++e) {
        int z[4] = {0, 0, 0, 0}, r = e;
        for (int a = s - 1; a >= 0; --a) {
            z[a] = r % li.D;
            r /= li.D;
        }
        if (member(z)) li.cosets.push_back({z[0], z[1], z[2], z[3]});
    }
    return true;
}

std::vector<std::vector<int>> canonical_columns(int s, const int *xi, int n)
{
    std::vector<std::vector<int>> cols;
    for (int j = 0; j < n; ++j) {
        std::vector<int> c(s);
        for (int a = 0; a < s; ++a) c[a] = xi[a * n + j];
        int sg = 0;
        for (int a = 0; a < s && !sg; ++a) sg = (c[a] > 0) - (c[a] < 0);
        if (sg < 0)
            for (int &v : c) v = -v;
        cols.push_back(c);
    }
    std::sort(cols.begin(), cols.end());
    return cols;
}

interp_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return INTERP_OK;
    if (e == cudaErrorMemoryAllocation) return INTERP_ENOMEM;
    return INTERP_ECUDA;
}

// every device allocation call of the library goes through these (counted for
// interp_debug_device_allocations)
std::atomic<long long> g_dev_allocs{0};

template <class T>
cudaError_t lib_malloc(T **p, size_t bytes)
{
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

template <class T>
cudaError_t lib_malloc_async(T **p, size_t bytes, cudaStream_t st)
{
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocAsync(reinterpret_cast<void **>(p), bytes, st);
}

}  // namespace

// ------------------------------------------------------------------------------------ the handle

// Gradient scratch of interp_backward_noalloc: a file-scope device array, so that entry point
// allocates nothing.  Host code must not use the name as a pointer: the device address comes from
// cudaGetSymbolAddress, looked up once per device and cached below.
static __device__ __align__(256) float g_noalloc_scratch[INTERP_NOALLOC_MAX_GRAD_ELEMS];

namespace {
constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (set up on the first call there)
interp_status noalloc_scratch(int dev, float **out)
{
    if (dev < 0 || dev >= kMaxDevices) return INTERP_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        float *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return INTERP_ECUDA;
        }
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return INTERP_OK;
}
}  // namespace

struct interp {
    const SplineOps *ops = nullptr;
    int s = 0;
    int dims[4] = {1, 1, 1, 1};
    ibl::Layout lay{};         // layout of the stored coefficients (storage element size)
    ibl::Layout lay32{};       // FP32 layout of the adjoint's padded gradient buffer
    int64_t coeff_count = 0;   // unpadded elements over all cosets
    interp_dtype storage = INTERP_F32;
    void *coeffs = nullptr;    // padded, bricked storage
    float *dpad = nullptr;     // padded FP32 gradient buffer (allocated by the first interp_backward)
    int device = 0;
    int sms = 148;                  // SMs of the handle's device (grid caps)
    // launch options (interp_set_option; initial values from the environment at creation):
    // -1 = the measured default
    int opt_binned = -1;            // piece-binned kernels for multi-piece splines: 0 / 1
    int opt_presort = -1;           // the piece pre-sort: 0 / 1 for any multi-piece spline and call size
    int opt_bin_small = 0;          // binned kernels on 256-query tiles: 0 / 1
    int opt_dense = -1;             // dense piece tables: 0 / 1
    int opt_adjoint_bins = -1;      // the adjoint on spatially binned queries: 0 / 1
    unsigned *sort_keys = nullptr;  // interp_sort_points bin counters
    int sort_nkeys = 0;
    // interp_eval_host staging: kHostSlots slots of (points, values, gradients), one stream each
    static constexpr int kHostSlots = 2;
    float *stage[kHostSlots] = {};
    cudaStream_t hs[kHostSlots] = {};
    cudaEvent_t hev[kHostSlots + 1] = {};
};

// ------------------------------------------------------------------------------------ piece pre-sort
//
// The piece-binned kernels sort a tile's (query, coset) items by piece (Sec. 4.3's sub-regions)
// in shared memory, but a tile of random queries still meets every piece, so each tile streams
// the code of all K unrolled pieces.  Where those pieces together far exceed the instruction
// caches (BCC V_2: 14 pieces of ~1000 immediate FMAs per coset), the queries are first sorted
// across the whole call by the pieces of their first cosets (a device-wide counting sort), the
// binned kernel runs on the sorted points, and the results go back to the callers' positions.
// A query's sum does not depend on which other queries share its tile, so the values are the
// binned kernel's bit for bit.  Scratch comes from a stream-ordered pool per call (calls on one
// handle may run concurrently on several streams); under stream capture, or when the scratch
// cannot be had, the call runs the binned kernel on the unsorted points instead.

namespace {

constexpr int kPsMaxKeys = 1024;           // keys: the pieces of the first c cosets, K^c <= 1024
constexpr int64_t kPsChunk = 1 << 22;      // queries sorted at a time (2^21 .. 2^23 measured: best value + grad)
constexpr int kPsBlock = 4096;             // queries per CTA of the scatter

// key of each query (mixed radix K over the pieces of its first c cosets) and the keys' totals
__global__ void __launch_bounds__(256) k_ps_count(const int32_t *__restrict__ piece, int n, int M, int c, int K,
                                                  int nkeys, uint16_t *__restrict__ key, unsigned *__restrict__ total)
{
    __shared__ unsigned hist[kPsMaxKeys];
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        unsigned k = 0;
        for (int j = 0; j < c; ++j) k = k * K + min((unsigned)piece[(int64_t)q * M + j], (unsigned)(K - 1));
        key[q] = (uint16_t)k;
        atomicAdd(&hist[k], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x)
        if (hist[i]) atomicAdd(&total[i], hist[i]);
}

// exclusive prefix sum of the totals into the cursors; zeroes the totals for the next chunk
__global__ void __launch_bounds__(kPsMaxKeys) k_ps_scan(unsigned *__restrict__ total, unsigned *__restrict__ cursor,
                                                         int nkeys)
{
    __shared__ unsigned s[kPsMaxKeys];
    const int t = threadIdx.x;
    const unsigned v = t < nkeys ? total[t] : 0u;
    s[t] = v;
    __syncthreads();
    for (int off = 1; off < kPsMaxKeys; off <<= 1) {
        const unsigned a = t >= off ? s[t - off] : 0u;
        __syncthreads();
        s[t] += a;
        __syncthreads();
    }
    if (t < nkeys) {
        cursor[t] = s[t] - v;
        total[t] = 0;
    }
}

// each CTA reserves, per key, a range of the chunk's sorted order for its kPsBlock queries and
// copies them there (a CTA-local sort before the copy, for contiguous stores, measured no faster)
template <int S>
__global__ void __launch_bounds__(256) k_ps_scatter(const float *__restrict__ pts, const float *__restrict__ gout,
                                                    const uint16_t *__restrict__ key, int n, int nkeys,
                                                    unsigned *__restrict__ cursor, int32_t *__restrict__ perm,
                                                    float *__restrict__ pts_s, float *__restrict__ gout_s)
{
    __shared__ unsigned cnt[kPsMaxKeys], base[kPsMaxKeys];
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const int q0 = blockIdx.x * kPsBlock, q1 = min(n, q0 + kPsBlock);
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) atomicAdd(&cnt[key[q]], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) {
        const unsigned c = cnt[i];
        base[i] = c ? atomicAdd(&cursor[i], c) : 0u;
        cnt[i] = 0;
    }
    __syncthreads();
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const unsigned k = key[q];
        const unsigned p = base[k] + atomicAdd(&cnt[k], 1u);
        perm[p] = q;
#pragma unroll
        for (int a = 0; a < S; ++a) pts_s[(int64_t)p * S + a] = pts[(int64_t)q * S + a];
        if (gout) gout_s[p] = gout[q];
    }
}

// results of the sorted queries back to their callers' positions
template <int S>
__global__ void __launch_bounds__(256) k_ps_unpermute(const int32_t *__restrict__ perm, int n,
                                                      const float *__restrict__ out_s, const float *__restrict__ grad_s,
                                                      float *__restrict__ out, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int q = perm[i];
    if (out) out[q] = out_s[i];
    if (grad) {
#pragma unroll
        for (int a = 0; a < S; ++a) grad[(int64_t)q * S + a] = grad_s[(int64_t)i * S + a];
    }
}

std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

// the per-device pool of the pre-sort scratch (kept up to 1 GiB between calls)
cudaError_t ps_pool(int dev, cudaMemPool_t *out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps p = {};
        p.allocType = cudaMemAllocationTypePinned;
        p.location.type = cudaMemLocationTypeDevice;
        p.location.id = dev;
        cudaMemPool_t pool = nullptr;
        g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
        cudaError_t e = cudaMemPoolCreate(&pool, &p);
        if (e != cudaSuccess) return e;
        uint64_t keep = 1ull << 30;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// whether a call of npts queries (at least 2^16) takes the pre-sort.  Measured on 2^24 random
// queries, sort included: faster for many large pieces (K >= 8 pieces of >= 500 FMAs per coset:
// BCC V_2, value 5.76 -> 2.95 ms, value+grad 6.95 -> 3.61 ms, adjoint 7.88 -> 3.34 ms) and for
// the 8-coset D4 spline, whose gathers come from DRAM (value 19.3 -> 17.7 ms, value+grad
// 19.7 -> 16.6 ms); slower for D4* (value 3.37 -> 3.91 ms: its 6 pieces' code is amortised
// within the tiles already, the sort is not) and no faster for BCC V_1 or FCC V_2, whose pieces
// fit the instruction caches.  INTERP_B300_PRESORT=0 / 1 forces it off / on.
bool presort_default(const SplineOps *ops)
{
    return (ops->K >= 8 && ops->fma_value / ops->M >= 500.0) || (ops->M >= 8 && ops->K >= 4);
}

bool presort_wanted(const interp *h, int64_t npts)
{
    if (h->opt_presort >= 0) return h->opt_presort == 1;
    return npts >= (1 << 16) && presort_default(h->ops);
}

// the handle's launch options as the launchers' flags
int launch_flags(const interp *h)
{
    int f = 0;
    if (h->opt_bin_small == 1) f |= ibr::FLAG_BIN_SMALL;
    if (h->opt_dense == 1) f |= ibr::FLAG_DENSE_ON;
    if (h->opt_dense == 0) f |= ibr::FLAG_DENSE_OFF;
    if (h->opt_binned == 1) f |= ibr::FLAG_BINNED_ON;
    if (h->opt_binned == 0) f |= ibr::FLAG_BINNED_OFF;
    return f;
}

struct PresortWs {
    void *block = nullptr;
    int32_t *piece = nullptr, *perm = nullptr;
    uint16_t *key = nullptr;
    float *pts_s = nullptr, *gout_s = nullptr, *out_s = nullptr, *grad_s = nullptr;
    unsigned *total = nullptr, *cursor = nullptr;
    int c = 1, nkeys = 1;
};

// scratch for chunks of up to min(npts, kPsChunk) queries on `st`; false (error cleared) when the
// stream is capturing or the pool has no room
bool ps_acquire(const interp *h, int64_t npts, cudaStream_t st, PresortWs &w);
void ps_release(PresortWs &w, cudaStream_t st)
{
    if (w.block) cudaFreeAsync(w.block, st);
    w.block = nullptr;
}

// sort chunk [pts, pts + m) (and its gout) by key: fills w.perm, w.pts_s (and w.gout_s)
cudaError_t ps_sort_chunk(const interp *h, PresortWs &w, const float *pts, const float *gout, int m, cudaStream_t st);
cudaError_t ps_unpermute(int s, const PresortWs &w, int m, float *out, float *grad, cudaStream_t st)
{
    const unsigned grid = (unsigned)((m + 255) / 256);
    if (s == 3)
        k_ps_unpermute<3><<<grid, 256, 0, st>>>(w.perm, m, w.out_s, w.grad_s, out, grad);
    else
        k_ps_unpermute<4><<<grid, 256, 0, st>>>(w.perm, m, w.out_s, w.grad_s, out, grad);
    return cudaPeekAtLastError();
}

}  // namespace

// allow_presort = false: never the piece pre-sort (it takes scratch from the library's pool)
static cudaError_t eval_launch(const interp *h, const float *pts, int64_t npts, float *out, float *grad, const float *gout,
                               int mode, cudaStream_t st, bool allow_presort = true)
{
    const int dt = h->storage == INTERP_F32 ? 0 : (h->storage == INTERP_F16 ? 1 : 2);
    // splines whose pieces' divergent work is large (>= 4 pieces, >= 200 nonzeros of A_j in all:
    // D4*, BCC V_1 and V_2, FCC V_2) run the piece-binned kernel; for few or small pieces (FCC:
    // 3 pieces, FCC V_1: 74 nonzeros) the sort costs more than the divergence it removes
    // (measured; ops_inst.cu's binned_default).  The handle's "binned" option forces the plain /
    // binned kernel.
    const bool want = h->opt_binned >= 0 ? h->opt_binned == 1 : h->ops->binned_eval;
    const bool binned = want && h->ops->eval_binned[dt][mode];
    const ibr::EvalFn fn = (binned ? h->ops->eval_binned : h->ops->eval)[dt][mode];
    const int flags = launch_flags(h);
    PresortWs w;
    if (!binned || !allow_presort || !presort_wanted(h, npts) || !ps_acquire(h, npts, st, w))
        return fn(pts, npts, h->coeffs, h->lay, out, grad, gout, flags, st);
    const int s = h->s;
    cudaError_t e = cudaSuccess;
    for (int64_t q0 = 0; q0 < npts && e == cudaSuccess; q0 += kPsChunk) {
        const int m = (int)std::min<int64_t>(kPsChunk, npts - q0);
        e = ps_sort_chunk(h, w, pts + q0 * s, mode == 2 ? gout + q0 : nullptr, m, st);
        // value (and gradient) of the sorted queries; the pullback (mode 2) writes w * grad only
        if (e == cudaSuccess)
            e = fn(w.pts_s, m, h->coeffs, h->lay, mode == 2 ? nullptr : w.out_s, mode >= 1 ? w.grad_s : nullptr,
                   mode == 2 ? w.gout_s : nullptr, flags, st);
        if (e == cudaSuccess)
            e = ps_unpermute(s, w, m, mode == 2 || !out ? nullptr : out + q0, mode >= 1 ? grad + q0 * s : nullptr, st);
    }
    ps_release(w, st);
    return e;
}

// ------------------------------------------------------------------------------------ adjoint on spatial bins
//
// interp_backward on many queries of a 3-D spline with few pieces: a counting sort of the queries
// into bins of 2^box_lb coset-0 cells per axis (count, scan, scatter of (x, y, z, gout) records),
// then one work item per chunk of a bin, which sums its contributions in a shared-memory box and
// adds the box to the padded gradient buffer (ib::k_adjoint_box).  The scratch comes per call from
// the library's stream-ordered pool, as for the piece pre-sort.

namespace {

constexpr int kBoxChunk = 32768;          // queries per work item at most
constexpr int kBoxSharedBins = 8192;      // per-CTA bin counters in shared memory up to this many bins
constexpr int kBoxBlock = 4096;           // queries per CTA of the count and scatter kernels

struct BoxGeom {
    int D, H2, lb, nb[3], nbins;
};

__device__ __forceinline__ int box_key(const float *p, float w, const BoxGeom &g, const ibl::Layout &L)
{
    const float x[3] = {p[0], p[1], p[2]};
    return g.D == 2 ? ib::box_key3<2>(x, w, g.H2, L, g.lb, g.nb) : ib::box_key3<1>(x, w, g.H2, L, g.lb, g.nb);
}

// queries per thread and round of the count and scatter kernels (independent loads in flight)
constexpr int kBoxUnroll = 4;

__global__ void __launch_bounds__(256) k_box_count(const float *__restrict__ pts, const float *__restrict__ gout, int n,
                                                   BoxGeom g, ibl::Layout L, unsigned *__restrict__ counts,
                                                   int *__restrict__ keys, float4 *__restrict__ rec)
{
    __shared__ unsigned hist[kBoxSharedBins];
    const bool sh = g.nbins <= kBoxSharedBins;
    if (sh) {
        for (int i = threadIdx.x; i < g.nbins; i += blockDim.x) hist[i] = 0;
        __syncthreads();
    }
    const int q0 = blockIdx.x * kBoxBlock, q1 = min(n, q0 + kBoxBlock);
    for (int qb = q0 + threadIdx.x; qb < q1; qb += kBoxUnroll * blockDim.x) {
        int key[kBoxUnroll];
#pragma unroll
        for (int u = 0; u < kBoxUnroll; ++u) {
            const int q = qb + u * blockDim.x;
            key[u] = -1;
            if (q < q1) {
                const float *p = pts + (int64_t)q * 3;
                const float w = gout[q];
                key[u] = box_key(p, w, g, L);
                keys[q] = key[u];
                rec[q] = make_float4(p[0], p[1], p[2], w);     // the query as one 16-byte record
            }
        }
#pragma unroll
        for (int u = 0; u < kBoxUnroll; ++u) {
            // a warp whose queries all fall in one bin (sorted input) adds once; otherwise one
            // atomic per query (random keys rarely collide within a warp)
            const unsigned act = __activemask();
            const int k0 = __shfl_sync(act, key[u], __ffs(act) - 1);
            if (__all_sync(act, key[u] == k0)) {
                if (k0 >= 0 && (int)(threadIdx.x & 31) == __ffs(act) - 1)
                    atomicAdd(sh ? &hist[k0] : &counts[k0], (unsigned)__popc(act));
            } else if (key[u] >= 0) {
                atomicAdd(sh ? &hist[key[u]] : &counts[key[u]], 1u);
            }
        }
    }
    if (sh) {
        __syncthreads();
        for (int i = threadIdx.x; i < g.nbins; i += blockDim.x)
            if (hist[i]) atomicAdd(&counts[i], hist[i]);
    }
}

// one CTA: bin_start = exclusive prefix of the counts (nbins + 1 entries), item_start = exclusive
// prefix of the work items ceil(count / chunk), cursor = bin_start; counts reset to zero
__global__ void __launch_bounds__(1024) k_box_scan(unsigned *__restrict__ counts, int nbins, int chunk,
                                                   int *__restrict__ bin_start, int *__restrict__ item_start,
                                                   unsigned *__restrict__ cursor)
{
    __shared__ unsigned sq[1024], si[1024];
    const int t = threadIdx.x;
    const int per = (nbins + 1023) / 1024, b0 = min(nbins, t * per), b1 = min(nbins, b0 + per);
    unsigned cq = 0, ci = 0;
    for (int b = b0; b < b1; ++b) {
        cq += counts[b];
        ci += (counts[b] + chunk - 1) / chunk;
    }
    sq[t] = cq;
    si[t] = ci;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned aq = t >= off ? sq[t - off] : 0u, ai = t >= off ? si[t - off] : 0u;
        __syncthreads();
        sq[t] += aq;
        si[t] += ai;
        __syncthreads();
    }
    unsigned pq = sq[t] - cq, pi = si[t] - ci;
    for (int b = b0; b < b1; ++b) {
        const unsigned c = counts[b];
        bin_start[b] = (int)pq;
        item_start[b] = (int)pi;
        cursor[b] = pq;
        pq += c;
        pi += (c + chunk - 1) / chunk;
        counts[b] = 0;
    }
    if (t == 1023) {
        bin_start[nbins] = (int)sq[1023];
        item_start[nbins] = (int)si[1023];
    }
}

// each CTA reserves, per bin, a range of the sorted order for its kBoxBlock queries and writes
// their indices there (cnt / base: dynamic shared memory, 2 x nbins counters, when nbins <=
// kBoxSharedBins; else one global atomic per distinct key of a warp)
__global__ void __launch_bounds__(256) k_box_scatter(const int *__restrict__ keys, int n, int nbins,
                                                     unsigned *__restrict__ cursor, int *__restrict__ idx)
{
    extern __shared__ unsigned box_sh[];
    unsigned *cnt = box_sh, *base = box_sh + nbins;
    const bool sh = nbins <= kBoxSharedBins;
    const int q0 = blockIdx.x * kBoxBlock, q1 = min(n, q0 + kBoxBlock);
    const int lane = threadIdx.x & 31;
    if (sh) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        for (int qb = q0 + threadIdx.x; qb < q1; qb += kBoxUnroll * blockDim.x) {
            int key[kBoxUnroll];
#pragma unroll
            for (int u = 0; u < kBoxUnroll; ++u) {
                const int q = qb + u * blockDim.x;
                key[u] = q < q1 ? keys[q] : -1;
            }
#pragma unroll
            for (int u = 0; u < kBoxUnroll; ++u) {
                const unsigned act = __activemask();
                const int k0 = __shfl_sync(act, key[u], __ffs(act) - 1);
                if (__all_sync(act, key[u] == k0)) {
                    if (k0 >= 0 && lane == __ffs(act) - 1) atomicAdd(&cnt[k0], (unsigned)__popc(act));
                } else if (key[u] >= 0) {
                    atomicAdd(&cnt[key[u]], 1u);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
            const unsigned c = cnt[i];
            base[i] = c ? atomicAdd(&cursor[i], c) : 0u;
            cnt[i] = 0;
        }
        __syncthreads();
    }
    for (int qb = q0 + threadIdx.x; qb < q1; qb += kBoxUnroll * blockDim.x) {
        int key[kBoxUnroll];
#pragma unroll
        for (int u = 0; u < kBoxUnroll; ++u) {
            const int q = qb + u * blockDim.x;
            key[u] = q < q1 ? keys[q] : -1;
        }
        unsigned pos[kBoxUnroll];
#pragma unroll
        for (int u = 0; u < kBoxUnroll; ++u) {
            // a warp whose queries all fall in one bin reserves its slots with one atomic;
            // otherwise each query takes its own slot
            const unsigned act = __activemask();
            const int leader = __ffs(act) - 1;
            const int k0 = __shfl_sync(act, key[u], leader);
            if (__all_sync(act, key[u] == k0)) {
                unsigned first = 0;
                if (k0 >= 0 && lane == leader) {
                    const unsigned c = (unsigned)__popc(act);
                    first = sh ? base[k0] + atomicAdd(&cnt[k0], c) : atomicAdd(&cursor[k0], c);
                }
                pos[u] = __shfl_sync(act, first, leader) + (unsigned)__popc(act & ((1u << lane) - 1u));
            } else {
                pos[u] = key[u] >= 0 ? (sh ? base[key[u]] + atomicAdd(&cnt[key[u]], 1u) : atomicAdd(&cursor[key[u]], 1u))
                                     : 0u;
            }
        }
#pragma unroll
        for (int u = 0; u < kBoxUnroll; ++u)
            if (key[u] >= 0) idx[pos[u]] = qb + u * (int)blockDim.x;
    }
}

// the scatter's dynamic shared memory above 48 KB (set once per device)
cudaError_t box_scatter_smem_optin(int dev)
{
    static std::mutex mu;
    static unsigned long long done = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && (done >> dev & 1ull)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k_box_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(2 * kBoxSharedBins * sizeof(unsigned)));
    if (e == cudaSuccess && dev >= 0 && dev < 64) done |= 1ull << dev;
    return e;
}

// the geometry of the bins for handle h, and whether a call of npts queries takes the binned adjoint
bool box_plan(const interp *h, int64_t npts, BoxGeom &g)
{
    const SplineOps *o = h->ops;
    if (!o->adjoint_box || h->opt_adjoint_bins == 0 || npts > INT32_MAX) return false;
    g.D = o->D;
    g.H2 = 2 * o->halo;
    g.lb = o->box_lb;
    int64_t nb = 1;
    for (int a = 0; a < 3; ++a) {
        g.nb[a] = (h->lay32.pdims[a] + (1 << g.lb) - 1) >> g.lb;
        nb *= g.nb[a];
    }
    if (nb > (1 << 24)) return false;
    g.nbins = (int)nb;
    if (h->opt_adjoint_bins == 1) return true;
    // worth it for wide stencils (>= 24 lookups per query) when the contributions outnumber the
    // boxes' global atomics at least four times (every bin's box of M (2^lb + 2 halo + 2)^3 sites
    // is added once).  Measured, 2^24 random queries: BCC quintic (32 lookups) 2.49 -> 1.46 ms,
    // CC 7-direction (53) 4.11 -> 3.52 ms; FCC 6-direction (16) 1.31 -> 1.51 ms, so narrow
    // stencils keep the one-atomic-per-contribution scatter
    const int W = (1 << g.lb) + g.H2 + 2;
    const double box_sites = (double)o->M * W * W * W;
    return o->lookups >= 24.0 && (double)npts * o->lookups >= 4.0 * (double)g.nbins * box_sites;
}

}  // namespace

// dL/dc into h->dpad on spatially binned queries; false (nothing enqueued, error cleared) when the
// scratch cannot be had or the stream is capturing
static bool adjoint_box_launch(const interp *h, const BoxGeom &g, const float *pts, int64_t npts, const float *gout,
                               cudaStream_t st, cudaError_t &err)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    const int n = (int)npts;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t nb = (size_t)g.nbins;
    const size_t sz[] = {up((size_t)n * 4), up((size_t)n * 4), up(nb * 4), up((nb + 1) * 4), up((nb + 1) * 4),
                         up(nb * 4), up((size_t)n * 16)};
    size_t bytes = 0;
    for (size_t b : sz) bytes += b;
    cudaMemPool_t pool = nullptr;
    void *block = nullptr;
    if (ps_pool(h->device, &pool) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    if (cudaMallocFromPoolAsync(&block, bytes, pool, st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    unsigned char *p = static_cast<unsigned char *>(block);
    int *keys = reinterpret_cast<int *>(p);
    p += sz[0];
    int *idx = reinterpret_cast<int *>(p);
    p += sz[1];
    unsigned *counts = reinterpret_cast<unsigned *>(p);
    p += sz[2];
    int *bin_start = reinterpret_cast<int *>(p);
    p += sz[3];
    int *item_start = reinterpret_cast<int *>(p);
    p += sz[4];
    unsigned *cursor = reinterpret_cast<unsigned *>(p);
    p += sz[5];
    float4 *rec = reinterpret_cast<float4 *>(p);
    cudaError_t e = cudaMemsetAsync(counts, 0, nb * 4, st);
    const unsigned grid = (unsigned)((n + kBoxBlock - 1) / kBoxBlock);
    const size_t scat_smem = g.nbins <= kBoxSharedBins ? 2 * nb * sizeof(unsigned) : 0;
    if (e == cudaSuccess && scat_smem > 48 * 1024) e = box_scatter_smem_optin(h->device);
    if (e == cudaSuccess) {
        k_box_count<<<grid, 256, 0, st>>>(pts, gout, n, g, h->lay32, counts, keys, rec);
        k_box_scan<<<1, 1024, 0, st>>>(counts, g.nbins, kBoxChunk, bin_start, item_start, cursor);
        k_box_scatter<<<grid, 256, scat_smem, st>>>(keys, n, g.nbins, cursor, idx);
        e = cudaPeekAtLastError();
    }
    if (e == cudaSuccess) {
        ibr::BoxArgs a;
        a.rec = reinterpret_cast<const float *>(rec);
        a.idx = idx;
        a.bin_start = bin_start;
        a.item_start = item_start;
        a.nbins = g.nbins;
        for (int i = 0; i < 3; ++i) a.nb[i] = g.nb[i];
        a.chunk = kBoxChunk;
        a.max_items = g.nbins + (n + kBoxChunk - 1) / kBoxChunk;
        a.lb = g.lb;
        e = h->ops->adjoint_box(a, h->lay32, h->dpad, st);
    }
    cudaFreeAsync(block, st);
    err = e;
    return true;
}

// dL/dc into h->dpad: the binned adjoint where it applies (3-D splines with few pieces, many
// queries); multi-piece splines with large pieces take the pre-sort like eval_launch (the
// adjoint's atomic scatter has no fixed summation order either way)
static cudaError_t adjoint_launch(const interp *h, const float *pts, int64_t npts, const float *gout, cudaStream_t st)
{
    BoxGeom g;
    cudaError_t eb = cudaSuccess;
    if (box_plan(h, npts, g) && adjoint_box_launch(h, g, pts, npts, gout, st, eb)) return eb;
    PresortWs w;
    if (h->ops->K < 4 || !presort_wanted(h, npts) || !ps_acquire(h, npts, st, w))
        return h->ops->adjoint(pts, npts, gout, h->lay32, h->dpad, st);
    const int s = h->s;
    cudaError_t e = cudaSuccess;
    for (int64_t q0 = 0; q0 < npts && e == cudaSuccess; q0 += kPsChunk) {
        const int m = (int)std::min<int64_t>(kPsChunk, npts - q0);
        e = ps_sort_chunk(h, w, pts + q0 * s, gout + q0, m, st);
        if (e == cudaSuccess) e = h->ops->adjoint(w.pts_s, m, w.gout_s, h->lay32, h->dpad, st);
    }
    ps_release(w, st);
    return e;
}

namespace {

bool ps_acquire(const interp *h, int64_t npts, cudaStream_t st, PresortWs &w)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    const SplineOps *ops = h->ops;
    w.c = 1;
    w.nkeys = ops->K;
    while (w.c < ops->M && w.nkeys * ops->K <= kPsMaxKeys) {
        ++w.c;
        w.nkeys *= ops->K;
    }
    if (w.nkeys > kPsMaxKeys) return false;
    const size_t C = (size_t)std::min<int64_t>(npts, kPsChunk), s = (size_t)h->s;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t sz[] = {up(C * ops->M * 4), up(C * 2), up(C * 4), up(C * s * 4), up(C * 4), up(C * 4),
                         up(C * s * 4), up((size_t)kPsMaxKeys * 4), up((size_t)kPsMaxKeys * 4)};
    size_t bytes = 0;
    for (size_t b : sz) bytes += b;
    cudaMemPool_t pool = nullptr;
    if (ps_pool(h->device, &pool) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    if (cudaMallocFromPoolAsync(&w.block, bytes, pool, st) != cudaSuccess) {
        cudaGetLastError();
        w.block = nullptr;
        return false;
    }
    unsigned char *p = static_cast<unsigned char *>(w.block);
    void **dst[] = {(void **)&w.piece, (void **)&w.key,   (void **)&w.perm,  (void **)&w.pts_s, (void **)&w.gout_s,
                    (void **)&w.out_s, (void **)&w.grad_s, (void **)&w.total, (void **)&w.cursor};
    for (int i = 0; i < 9; ++i) {
        *dst[i] = p;
        p += sz[i];
    }
    if (cudaMemsetAsync(w.total, 0, (size_t)kPsMaxKeys * 4, st) != cudaSuccess) {
        cudaGetLastError();
        ps_release(w, st);
        return false;
    }
    return true;
}

cudaError_t ps_sort_chunk(const interp *h, PresortWs &w, const float *pts, const float *gout, int m, cudaStream_t st)
{
    const SplineOps *ops = h->ops;
    cudaError_t e = ops->debug(pts, m, h->lay32, nullptr, w.piece, st);
    if (e != cudaSuccess) return e;
    const unsigned gc = (unsigned)std::min<int64_t>((m + 255) / 256, (int64_t)h->sms * 8);
    k_ps_count<<<gc, 256, 0, st>>>(w.piece, m, ops->M, w.c, ops->K, w.nkeys, w.key, w.total);
    k_ps_scan<<<1, kPsMaxKeys, 0, st>>>(w.total, w.cursor, w.nkeys);
    const unsigned gs = (unsigned)((m + kPsBlock - 1) / kPsBlock);
    if (h->s == 3)
        k_ps_scatter<3><<<gs, 256, 0, st>>>(pts, gout, w.key, m, w.nkeys, w.cursor, w.perm, w.pts_s, w.gout_s);
    else
        k_ps_scatter<4><<<gs, 256, 0, st>>>(pts, gout, w.key, m, w.nkeys, w.cursor, w.perm, w.pts_s, w.gout_s);
    return cudaPeekAtLastError();
}

}  // namespace

// the handle for a registry entry: validate dims and storage, lay out and zero the padded arrays
static interp_status create_handle(const SplineOps *ops, const int32_t *dims, interp_dtype storage, interp_t **out)
{
    const int s = ops->s;
    if (storage != INTERP_F32 && storage != INTERP_F16 && storage != INTERP_BF16) return INTERP_EINVAL;
    for (int a = 0; a < s; ++a)
        if (dims[a] < 1) return INTERP_EINVAL;
    if (storage != INTERP_F32 && !ops->eval[storage == INTERP_F16 ? 1 : 2][0]) return INTERP_EUNSUPPORTED;

    interp *h = new (std::nothrow) interp;
    if (!h) return INTERP_ENOMEM;
    h->ops = ops;
    h->s = s;
    h->storage = storage;
    const int pad = 2 * ops->halo;
    int64_t cc = 1;
    for (int a = 0; a < s; ++a) {
        h->dims[a] = dims[a];
        cc *= dims[a];
    }
    const int esz = storage == INTERP_F32 ? 4 : 2;
    // cosets in separate bricked arrays (the kernels' brick widths are compile-time constants of
    // this layout; cosets side by side inside the bricks measured slower on the BCC quintic
    // workload: 15.1 against 13.4 L1 misses per query)
    if (!ibl::make_layout(h->lay, s, h->dims, pad, esz, ops->M, false) ||
        !ibl::make_layout(h->lay32, s, h->dims, pad, 4, ops->M, false)) {
        delete h;
        return INTERP_ESIZE;
    }
    h->coeff_count = cc * ops->M;
    cudaGetDevice(&h->device);
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || h->sms < 1) {
        cudaGetLastError();
        h->sms = 148;
    }
    // initial launch options from the environment (read once, here)
    auto env01 = [](const char *name) {
        const char *e = std::getenv(name);
        return e ? (e[0] == '1' ? 1 : 0) : -1;
    };
    h->opt_binned = env01("INTERP_B300_BINNED");
    h->opt_presort = env01("INTERP_B300_PRESORT");
    h->opt_dense = env01("INTERP_B300_DENSE");
    h->opt_adjoint_bins = env01("INTERP_B300_ADJOINT_BINS");
    if (const char *e = std::getenv("INTERP_B300_BINCFG")) h->opt_bin_small = e[0] == 's' ? 1 : 0;
    const size_t bytes = (size_t)h->lay.total * esz;
    cudaError_t e = lib_malloc(&h->coeffs, bytes);
    if (e == cudaSuccess) e = cudaMemset(h->coeffs, 0, bytes);
    if (e != cudaSuccess) {
        cudaFree(h->coeffs);
        delete h;
        cudaGetLastError();
        return cuda_status(e);
    }
    *out = h;
    return INTERP_OK;
}

extern "C" {

const char *interp_strerror(interp_status st)
{
    switch (st) {
    case INTERP_OK: return "ok";
    case INTERP_EINVAL: return "invalid argument";
    case INTERP_EUNSUPPORTED: return "unsupported lattice/spline (no generated tables) or dimension";
    case INTERP_ENOMEM: return "out of memory";
    case INTERP_ECUDA: return "CUDA error";
    case INTERP_ESIZE: return "size exceeds a documented limit";
    }
    return "unknown status";
}

int interp_num_splines(void) { return (int)registry().size(); }

long long interp_debug_device_allocations(void) { return g_dev_allocs.load(std::memory_order_relaxed); }

const char *interp_spline_name(int i)
{
    if (i < 0 || i >= (int)registry().size()) return nullptr;
    return registry()[i].name;
}

const char *interp_table_digest(void) { return INTERP_GEN_DIGEST; }

interp_status interp_create(int s, const int32_t *L, const int32_t *xi, int n, const int32_t *dims,
                            interp_dtype storage, interp_t **out)
{
    if (!out) return INTERP_EINVAL;
    *out = nullptr;
    if (!L || !xi || !dims || n < 1) return INTERP_EINVAL;
    if (s < 3 || s > 4) return INTERP_EUNSUPPORTED;
    if (storage != INTERP_F32 && storage != INTERP_F16 && storage != INTERP_BF16) return INTERP_EINVAL;
    for (int a = 0; a < s; ++a)
        if (dims[a] < 1) return INTERP_EINVAL;
    LatticeInfo li;
    if (!lattice_info(s, L, li)) return INTERP_EINVAL;
    const auto want = canonical_columns(s, xi, n);
    const SplineOps *ops = nullptr;
    for (const auto &o : registry()) {
        // box splines only: a Voronoi spline's recorded generators are not a direction matrix
        if (o.kind != 0 || o.s != s || o.nxi != n || o.D != li.D || o.M != (int)li.cosets.size()) continue;
        if (canonical_columns(s, o.xi, o.nxi) != want) continue;
        bool same = true;
        for (int k = 0; k < o.M && same; ++k)
            for (int a = 0; a < s; ++a) same &= o.cosets[k * s + a] == li.cosets[k][a];
        if (same) {
            ops = &o;
            break;
        }
    }
    if (!ops) return INTERP_EUNSUPPORTED;
    return create_handle(ops, dims, storage, out);
}

interp_status interp_create_named(const char *spline, const int32_t *dims, interp_dtype storage, interp_t **out)
{
    if (!out) return INTERP_EINVAL;
    *out = nullptr;
    if (!spline || !dims) return INTERP_EINVAL;
    for (const auto &o : registry())
        if (std::strcmp(o.name, spline) == 0) return create_handle(&o, dims, storage, out);
    return INTERP_EUNSUPPORTED;
}

void interp_destroy(interp_t *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->coeffs);
    cudaFree(h->dpad);
    cudaFree(h->sort_keys);
    for (int i = 0; i < interp::kHostSlots; ++i) {
        cudaFree(h->stage[i]);
        if (h->hs[i]) cudaStreamDestroy(h->hs[i]);
    }
    for (auto &ev : h->hev)
        if (ev) cudaEventDestroy(ev);
    delete h;
}

interp_status interp_info(const interp_t *h, interp_info_t *info)
{
    if (!h || !info) return INTERP_EINVAL;
    std::memset(info, 0, sizeof(*info));
    const SplineOps &o = *h->ops;
    info->s = o.s;
    info->n_cosets = o.M;
    info->D = o.D;
    info->halo = o.halo;
    info->n_pieces = o.K;
    info->degree = o.deg;
    info->n_monomials = o.nmon;
    for (int a = 0; a < 4; ++a) info->dims[a] = a < o.s ? h->dims[a] : 1;
    for (int k = 0; k < o.M && k < 8; ++k)
        for (int a = 0; a < o.s; ++a) info->cosets[k][a] = o.cosets[k * o.s + a];
    info->lookups_per_query = o.lookups;
    info->fma_value_per_query = o.fma_value;
    info->fma_grad_per_query = o.fma_grad;
    info->coeff_count = h->coeff_count;
    info->name = o.name;
    info->kind = o.kind;
    info->presort = presort_default(&o) ? 1 : 0;
    info->binned = o.binned_eval ? 1 : 0;
    info->coop = o.coop_eval ? 1 : 0;
    return INTERP_OK;
}

interp_status interp_set_option(interp_t *h, const char *name, int value)
{
    if (!h || !name) return INTERP_EINVAL;
    int *slot = nullptr;
    int lo = -1;
    if (std::strcmp(name, "binned") == 0) slot = &h->opt_binned;
    else if (std::strcmp(name, "presort") == 0) slot = &h->opt_presort;
    else if (std::strcmp(name, "dense") == 0) slot = &h->opt_dense;
    else if (std::strcmp(name, "adjoint_bins") == 0) slot = &h->opt_adjoint_bins;
    else if (std::strcmp(name, "bin_small_tiles") == 0) {
        slot = &h->opt_bin_small;
        lo = 0;
    }
    if (!slot || value < lo || value > 1) return INTERP_EINVAL;
    *slot = value;
    return INTERP_OK;
}

interp_status interp_get_option(const interp_t *h, const char *name, int *value)
{
    if (!h || !name || !value) return INTERP_EINVAL;
    if (std::strcmp(name, "binned") == 0) *value = h->opt_binned;
    else if (std::strcmp(name, "presort") == 0) *value = h->opt_presort;
    else if (std::strcmp(name, "dense") == 0) *value = h->opt_dense;
    else if (std::strcmp(name, "adjoint_bins") == 0) *value = h->opt_adjoint_bins;
    else if (std::strcmp(name, "bin_small_tiles") == 0) *value = h->opt_bin_small;
    else return INTERP_EINVAL;
    return INTERP_OK;
}

interp_status interp_prefilter(interp_t *h, const float *samples, int ntaps, const int32_t *taps, const float *weights,
                               void *stream)
{
    if (!h || !samples || !taps || !weights || ntaps < 1 || ntaps > kMaxTaps) return INTERP_EINVAL;
    const SplineOps &o = *h->ops;
    const int s = o.s, M = o.M, D = o.D;
    PrefilterTaps tp{};
    tp.ntaps = ntaps;
    for (int t = 0; t < ntaps; ++t) {
        tp.w[t] = weights[t];
        for (int a = 0; a < s; ++a)
            if (taps[t * s + a] < -64 || taps[t * s + a] > 64) return INTERP_EINVAL;
        // l_k + v lies on coset k' at index shift (l_k + v - l_k') / D; no coset: v is not a
        // lattice vector
        for (int k = 0; k < M; ++k) {
            int kk = -1;
            for (int c = 0; c < M && kk < 0; ++c) {
                bool same = true;
                for (int a = 0; a < s; ++a) {
                    const int u = o.cosets[k * s + a] + taps[t * s + a] - o.cosets[c * s + a];
                    same &= ((u % D) + D) % D == 0;
                }
                if (same) kk = c;
            }
            if (kk < 0) return INTERP_EINVAL;
            tp.src[k][t] = (signed char)kk;
            for (int a = 0; a < s; ++a)
                tp.shift[k][t][a] = (signed char)((o.cosets[k * s + a] + taps[t * s + a] - o.cosets[kk * s + a]) / D);
        }
    }
    // linear offsets of the taps in the sample array, and the reach of the filter
    int64_t stride[4] = {0, 0, 0, 0}, coset_stride = 1;
    for (int a = s - 1; a >= 0; --a) {
        stride[a] = coset_stride;
        coset_stride *= h->dims[a];
    }
    for (int k = 0; k < M; ++k)
        for (int t = 0; t < ntaps; ++t) {
            int64_t d = (int64_t)(tp.src[k][t] - k) * coset_stride;
            for (int a = 0; a < s; ++a) {
                d += tp.shift[k][t][a] * stride[a];
                tp.reach = std::max(tp.reach, (int)std::abs(tp.shift[k][t][a]));
                if (tp.shift[k][t][a] < 0) tp.neg[k][t] |= (unsigned char)(1u << a);
                if (tp.shift[k][t][a] > 0) tp.pos[k][t] |= (unsigned char)(1u << a);
            }
            tp.delta[k][t] = (int)d;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nl = h->dims[s - 1];
    const int runs = (nl + PF_RUN - 1) / PF_RUN;     // threads per row
    int lw = 0;
    while ((1 << lw) < runs && lw < 8) ++lw;
    const int chunks = (runs + 255) / 256;
    const int nrows = (int)(h->coeff_count / M / nl);
    const int rows_per_cta = chunks == 1 ? 256 >> lw : 1;
    const unsigned grid = chunks == 1 ? (unsigned)((nrows + rows_per_cta - 1) / rows_per_cta)
                                      : (unsigned)((int64_t)nrows * chunks);
    const unsigned threads = chunks == 1 ? (unsigned)(rows_per_cta << lw) : 256u;
    switch (h->storage) {
    case INTERP_F32:
        k_prefilter<float><<<grid, threads, 0, st>>>(samples, static_cast<float *>(h->coeffs), h->lay, lw, chunks,
                                                     nrows, M, (int)coset_stride, tp);
        break;
    case INTERP_F16:
        k_prefilter<__half><<<grid, threads, 0, st>>>(samples, static_cast<__half *>(h->coeffs), h->lay, lw, chunks,
                                                      nrows, M, (int)coset_stride, tp);
        break;
    default:
        k_prefilter<__nv_bfloat16><<<grid, threads, 0, st>>>(samples, static_cast<__nv_bfloat16 *>(h->coeffs), h->lay,
                                                             lw, chunks, nrows, M, (int)coset_stride, tp);
        break;
    }
    return cuda_status(cudaPeekAtLastError());
}

interp_status interp_set_coeffs(interp_t *h, const void *src, interp_dtype src_dtype, int src_on_device, void *stream)
{
    if (!h || !src) return INTERP_EINVAL;
    if (src_dtype < INTERP_F32 || src_dtype > INTERP_F64) return INTERP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t ssz = src_dtype == INTERP_F64 ? 8 : (src_dtype == INTERP_F32 ? 4 : 2);
    const size_t bytes = (size_t)h->coeff_count * ssz;
    const void *dsrc = src;
    void *tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!src_on_device) {
        e = lib_malloc_async(&tmp, bytes, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            if (tmp) cudaFreeAsync(tmp, st);
            cudaGetLastError();
            return cuda_status(e);
        }
        dsrc = tmp;
    }
    const unsigned grid = (unsigned)std::min<int64_t>((h->coeff_count + 255) / 256, (int64_t)h->sms * 32);
#define PADCOPY(ST, CT) \
    k_pad_copy<ST, CT><<<grid, 256, 0, st>>>(static_cast<const ST *>(dsrc), static_cast<CT *>(h->coeffs), h->coeff_count, h->lay)
#define PADCOPY_SRC(CT)                                              \
    switch (src_dtype) {                                             \
    case INTERP_F32: PADCOPY(float, CT); break;                      \
    case INTERP_F16: PADCOPY(__half, CT); break;                     \
    case INTERP_BF16: PADCOPY(__nv_bfloat16, CT); break;             \
    case INTERP_F64: PADCOPY(double, CT); break;                     \
    }
    switch (h->storage) {
    case INTERP_F32: PADCOPY_SRC(float); break;
    case INTERP_F16: PADCOPY_SRC(__half); break;
    case INTERP_BF16: PADCOPY_SRC(__nv_bfloat16); break;
    default: break;
    }
#undef PADCOPY_SRC
#undef PADCOPY
    e = cudaPeekAtLastError();
    if (tmp) {
        cudaError_t e2 = cudaFreeAsync(tmp, st);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

static interp_status eval_common(const interp_t *h, const float *pts, int64_t npts, float *out, float *grad,
                                 const float *gout, int mode, void *stream)
{
    if (!h || npts < 0) return INTERP_EINVAL;
    if (npts == 0) return INTERP_OK;
    if (!pts) return INTERP_EINVAL;
    if (mode == 0 && !out) return INTERP_EINVAL;
    if (mode >= 1 && !grad) return INTERP_EINVAL;
    if (mode == 2 && !gout) return INTERP_EINVAL;
    if (npts > (int64_t)INT32_MAX * kTPB) return INTERP_ESIZE;
    cudaError_t e = eval_launch(h, pts, npts, out, grad, gout, mode, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_eval(const interp_t *h, const float *pts, int64_t npts, float *out, void *stream)
{
    return eval_common(h, pts, npts, out, nullptr, nullptr, 0, stream);
}

interp_status interp_eval_grad(const interp_t *h, const float *pts, int64_t npts, float *out, float *grad, void *stream)
{
    return eval_common(h, pts, npts, out, grad, nullptr, 1, stream);
}

interp_status interp_eval_host(interp_t *h, const float *pts, int64_t npts, float *out, float *grad, void *stream)
{
    if (!h || npts < 0) return INTERP_EINVAL;
    if (npts == 0) return INTERP_OK;
    if (!pts || !out) return INTERP_EINVAL;
    // chunks of 2^20 queries rotate over kHostSlots streams: a slot's upload waits only for that
    // slot's previous download, so uploads, evaluations and downloads of neighbouring chunks
    // overlap (measured on the BCC quintic workload: two slots of 2^20 queries 6.54 ms per 2^24
    // queries, three of 2^19 6.77 ms; both directions' copies at once are the bound)
    constexpr int64_t kChunk = 1 << 20;
    constexpr int NS = interp::kHostSlots;
    const int s = h->s;
    const int64_t slot_floats = kChunk * (s + 1 + s);     // points, values, gradients
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < NS && e == cudaSuccess; ++i) {
        if (!h->stage[i]) e = lib_malloc(&h->stage[i], (size_t)slot_floats * sizeof(float));
        if (e == cudaSuccess && !h->hs[i]) e = cudaStreamCreateWithFlags(&h->hs[i], cudaStreamNonBlocking);
    }
    for (int i = 0; i < NS + 1 && e == cudaSuccess; ++i)
        if (!h->hev[i]) e = cudaEventCreateWithFlags(&h->hev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the internal streams start after the work already on `stream`
    e = cudaEventRecord(h->hev[NS], st);
    for (int i = 0; i < NS && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(h->hs[i], h->hev[NS], 0);
    int64_t chunk = 0;
    for (int64_t q0 = 0; q0 < npts && e == cudaSuccess; q0 += kChunk, ++chunk) {
        const int slot = (int)(chunk % NS);
        cudaStream_t ss = h->hs[slot];
        const int64_t m = std::min<int64_t>(kChunk, npts - q0);
        float *dp = h->stage[slot], *dv = dp + kChunk * s, *dg = dv + kChunk;
        // stream order inside a slot keeps its buffers from being overwritten while in use
        e = cudaMemcpyAsync(dp, pts + q0 * s, (size_t)m * s * sizeof(float), cudaMemcpyHostToDevice, ss);
        if (e == cudaSuccess) e = eval_launch(h, dp, m, dv, grad ? dg : nullptr, nullptr, grad ? 1 : 0, ss);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out + q0, dv, (size_t)m * sizeof(float), cudaMemcpyDeviceToHost, ss);
        if (e == cudaSuccess && grad)
            e = cudaMemcpyAsync(grad + q0 * s, dg, (size_t)m * s * sizeof(float), cudaMemcpyDeviceToHost, ss);
    }
    // `stream` continues after every internal stream
    for (int i = 0; i < NS && e == cudaSuccess; ++i) {
        e = cudaEventRecord(h->hev[i], h->hs[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->hev[i], 0);
    }
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_backward(interp_t *h, const float *pts, int64_t npts, const float *gout, float *dcoeffs,
                              float *dpts, void *stream)
{
    if (!h || npts < 0) return INTERP_EINVAL;
    if (npts == 0) return INTERP_OK;
    if (!pts || !gout) return INTERP_EINVAL;
    if (npts > (int64_t)INT32_MAX * kTPB) return INTERP_ESIZE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dpts) {
        interp_status s2 = eval_common(h, pts, npts, nullptr, dpts, gout, 2, stream);
        if (s2 != INTERP_OK) return s2;
    }
    if (!dcoeffs) return INTERP_OK;
    cudaError_t e = cudaSuccess;
    const size_t dbytes = (size_t)h->lay32.total * sizeof(float);
    if (!h->dpad) {
        e = lib_malloc(&h->dpad, dbytes);
        if (e != cudaSuccess) {
            h->dpad = nullptr;
            cudaGetLastError();
            return cuda_status(e);
        }
    }
    e = cudaMemsetAsync(h->dpad, 0, dbytes, st);
    if (e == cudaSuccess) e = adjoint_launch(h, pts, npts, gout, st);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::min<int64_t>((h->coeff_count + 255) / 256, (int64_t)h->sms * 32);
        k_unpad_add<<<grid, 256, 0, st>>>(h->dpad, dcoeffs, h->coeff_count, h->lay32);
        e = cudaPeekAtLastError();
    }
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_eval_rays(const interp_t *h, const interp_rays_t *rays, int with_grad, float *out, float *pts_out,
                               void *stream)
{
    if (!h || !rays || !out) return INTERP_EINVAL;
    if (rays->width < 1 || rays->height < 1 || rays->steps < 1) return INTERP_EINVAL;
    if ((int64_t)rays->width * rays->height > (int64_t)INT32_MAX) return INTERP_ESIZE;
    if (h->s != 3 || h->storage != INTERP_F32 || !h->ops->rays[0]) return INTERP_EUNSUPPORTED;
    ibl::RayGeom rg;
    static_assert(sizeof(rg.origin) == sizeof(rays->origin), "ray geometry layout");
    std::memcpy(rg.origin, rays->origin, sizeof(rg.origin));
    std::memcpy(rg.du, rays->du, sizeof(rg.du));
    std::memcpy(rg.dv, rays->dv, sizeof(rg.dv));
    std::memcpy(rg.dir, rays->dir, sizeof(rg.dir));
    std::memcpy(rg.lo, rays->box_lo, sizeof(rg.lo));
    std::memcpy(rg.hi, rays->box_hi, sizeof(rg.hi));
    rg.width = rays->width;
    rg.height = rays->height;
    rg.steps = rays->steps;
    cudaError_t e = h->ops->rays[with_grad ? 1 : 0](rg, h->coeffs, h->lay, out, pts_out, launch_flags(h),
                                                      static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_backward_noalloc(interp_t *h, const float *pts, int64_t npts, const float *gout, float *dcoeffs,
                                      float *dpts, void *stream)
{
    if (!h || npts < 0) return INTERP_EINVAL;
    // the static array's limit concerns dL/dc only: a dpts-only call never touches it
    const int64_t need = (int64_t)h->lay32.total;
    if (dcoeffs && need > INTERP_NOALLOC_MAX_GRAD_ELEMS) return INTERP_ESIZE;
    if (npts == 0) return INTERP_OK;
    if (!pts || !gout) return INTERP_EINVAL;
    if (npts > (int64_t)INT32_MAX * kTPB) return INTERP_ESIZE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return INTERP_ECUDA;
    }
    if (dev != h->device) return INTERP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dpts) {
        // the pullback without the piece pre-sort, whose scratch comes from the library's pool
        const cudaError_t e2 = eval_launch(h, pts, npts, nullptr, dpts, gout, 2, st, false);
        if (e2 != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e2);
        }
    }
    if (!dcoeffs) return INTERP_OK;
    float *scratch = nullptr;
    interp_status st0 = noalloc_scratch(dev, &scratch);
    if (st0 != INTERP_OK) return st0;
    cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)need * sizeof(float), st);
    if (e == cudaSuccess) e = h->ops->adjoint(pts, npts, gout, h->lay32, scratch, st);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::min<int64_t>((h->coeff_count + 255) / 256, (int64_t)h->sms * 32);
        k_unpad_add<<<grid, 256, 0, st>>>(scratch, dcoeffs, h->coeff_count, h->lay32);
        e = cudaPeekAtLastError();
    }
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_sort_points(interp_t *h, const float *pts, int64_t npts, int32_t *perm, float *pts_sorted,
                                 void *stream)
{
    if (!h || npts < 0 || (!perm && !pts_sorted)) return INTERP_EINVAL;
    if (npts == 0) return INTERP_OK;
    if (!pts) return INTERP_EINVAL;
    if (npts > (int64_t)INT32_MAX) return INTERP_ESIZE;
    const int s = h->s;
    // bins of 2^bb padded cells per axis; Morton keys of `bits` bits per axis, at most 2^22 keys
    int bb = s == 3 ? 2 : 1, bits = 0;
    for (;;) {
        int maxnb = 1;
        for (int a = 0; a < s; ++a) maxnb = std::max(maxnb, (h->lay32.pdims[a] + (1 << bb) - 1) >> bb);
        bits = 0;
        while ((1 << bits) < maxnb) ++bits;
        if (bits * s <= 22) break;
        ++bb;
    }
    const int nkeys = 1 << (bits * s);
    cudaError_t e = cudaSuccess;
    if (h->sort_nkeys < nkeys) {
        cudaFree(h->sort_keys);
        h->sort_keys = nullptr;
        h->sort_nkeys = 0;
        // the counters, then one partial sum per 4096 counters for the scan
        e = lib_malloc(&h->sort_keys, ((size_t)nkeys + nkeys / 4096 + 1) * sizeof(unsigned));
        if (e != cudaSuccess) {
            h->sort_keys = nullptr;
            cudaGetLastError();
            return cuda_status(e);
        }
        h->sort_nkeys = nkeys;
    }
    e = h->ops->sort(pts, npts, h->lay32, bb, bits, h->sort_keys, nkeys, perm, pts_sorted,
                     static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_debug_indices(const interp_t *h, const float *pts, int64_t npts, int32_t *cells, int32_t *piece,
                                   void *stream)
{
    if (!h || npts < 0) return INTERP_EINVAL;
    if (npts == 0) return INTERP_OK;
    if (!pts) return INTERP_EINVAL;
    cudaError_t e = h->ops->debug(pts, npts, h->lay32, cells, piece, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}


}  // extern "C"

// ------------------------------------------------------------------------------------ batched evaluation

struct interp_batch {
    struct Group {
        std::vector<ibl::BatchVol> vols;
        ibl::BatchVol *d_vols = nullptr;
        int64_t total = 0;
        int grid = 0;
    };
    Group g[2];                                   // [0]: persistent-kernel handles, [1]: the others
    unsigned long long *d_counters = nullptr;     // one work counter per group
    std::vector<std::string> names[2];            // spline name of every volume, per group
    std::map<std::string, int> tiles;             // queries per tile, per spline
    std::vector<const interp *> own;              // handles evaluated by their own launch (group 1)
    cudaStream_t cs = nullptr;                    // private stream for graph capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;
    int device = 0;
};

namespace {

constexpr int kDefaultTile = 1024;

// recompute the tile prefixes and upload the descriptor tables (synchronous)
cudaError_t batch_upload(interp_batch *b)
{
    for (int gi = 0; gi < 2; ++gi) {
        auto &G = b->g[gi];
        int64_t first = 0;
        for (size_t v = 0; v < G.vols.size(); ++v) {
            G.vols[v].tile = gi == 0 ? b->tiles[b->names[gi][v]] : kDefaultTile;
            G.vols[v].first_tile = first;
            first += (G.vols[v].npts + G.vols[v].tile - 1) / G.vols[v].tile;
        }
        G.total = first;
        if (!G.vols.empty()) {
            cudaError_t e = cudaMemcpy(G.d_vols, G.vols.data(), G.vols.size() * sizeof(ibl::BatchVol),
                                       cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return e;
        }
    }
    b->dirty = true;
    return cudaSuccess;
}

// enqueue one batched evaluation: the handles of the persistent kernel's splines in one launch
// (counter reset + kernel); the others (4-D, and 3-D splines whose pieces or registers would
// slow the persistent kernel for everyone) as one evaluation launch each
cudaError_t batch_enqueue(interp_batch *b, cudaStream_t st)
{
    auto &G = b->g[0];
    if (G.total > 0) {
        cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess)
            e = ibr::batch_launch_3d(G.d_vols, (int)G.vols.size(), G.total, b->d_counters, G.grid, st);
        if (e != cudaSuccess) return e;
    }
    for (size_t v = 0; v < b->own.size(); ++v) {
        const ibl::BatchVol &bv = b->g[1].vols[v];
        if (bv.npts == 0) continue;
        cudaError_t e = eval_launch(b->own[v], bv.pts, bv.npts, bv.out, nullptr, nullptr, 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void batch_free_graph(interp_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

}  // namespace

extern "C" {

void interp_batch_destroy(interp_batch_t *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free_graph(b);
    for (auto &G : b->g) cudaFree(G.d_vols);
    cudaFree(b->d_counters);
    if (b->cs) cudaStreamDestroy(b->cs);
    delete b;
}

interp_status interp_batch_create(const interp_batch_item *items, int n, interp_batch_t **out)
{
    if (!out) return INTERP_EINVAL;
    *out = nullptr;
    if (!items || n < 1) return INTERP_EINVAL;
    interp_batch *b = new (std::nothrow) interp_batch;
    if (!b) return INTERP_ENOMEM;
    cudaGetDevice(&b->device);
    for (int i = 0; i < n; ++i) {
        const interp_batch_item &it = items[i];
        if (!it.vol || it.npts < 0 || (it.npts > 0 && (!it.pts || !it.out))) {
            delete b;
            return INTERP_EINVAL;
        }
        if (it.vol->storage != INTERP_F32) {
            delete b;
            return INTERP_EUNSUPPORTED;
        }
        const int kind = it.vol->s == 3 ? ibr::batch_kind_3d(it.vol->ops->name) : -1;
        const int gi = kind >= 0 ? 0 : 1;
        ibl::BatchVol bv{};
        bv.c = static_cast<const float *>(it.vol->coeffs);
        bv.pts = it.pts;
        bv.out = it.out;
        bv.npts = it.npts;
        bv.kind = kind >= 0 ? kind : 0;
        bv.tile = kDefaultTile;
        bv.L = it.vol->lay;
        b->g[gi].vols.push_back(bv);
        b->names[gi].push_back(it.vol->ops->name);
        if (gi == 0) b->tiles.emplace(it.vol->ops->name, kDefaultTile);
        else b->own.push_back(it.vol);
    }
    cudaError_t e = lib_malloc(&b->d_counters, 2 * sizeof(unsigned long long));
    for (int gi = 0; gi < 2 && e == cudaSuccess; ++gi) {
        auto &G = b->g[gi];
        if (G.vols.empty()) continue;
        e = lib_malloc(&G.d_vols, G.vols.size() * sizeof(ibl::BatchVol));
        if (e == cudaSuccess && gi == 0) e = ibr::batch_grid_3d(&G.grid);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = batch_upload(b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        interp_batch_destroy(b);
        return cuda_status(e);
    }
    *out = b;
    return INTERP_OK;
}

interp_status interp_batch_tile(const interp_batch_t *b, const char *spline, int *tile)
{
    if (!b || !spline || !tile) return INTERP_EINVAL;
    auto it = b->tiles.find(spline);
    if (it == b->tiles.end()) return INTERP_EINVAL;
    *tile = it->second;
    return INTERP_OK;
}

interp_status interp_batch_set_tile(interp_batch_t *b, const char *spline, int tile)
{
    if (!b || !spline || tile < 128 || tile % 128 != 0) return INTERP_EINVAL;
    auto it = b->tiles.find(spline);
    if (it == b->tiles.end()) return INTERP_EINVAL;
    it->second = tile;
    const cudaError_t e = batch_upload(b);
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_batch_autotune(interp_batch_t *b, void *stream)
{
    if (!b) return INTERP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    static const int cand[] = {256, 512, 1024, 2048, 4096, 8192};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<std::string> names;
    for (auto &kv : b->tiles) names.push_back(kv.first);
    for (const auto &name : names) {
        int best = b->tiles[name];
        float best_ms = 1e30f;
        for (int t : cand) {
            if (e != cudaSuccess) break;
            b->tiles[name] = t;
            e = batch_upload(b);
            if (e == cudaSuccess) e = batch_enqueue(b, st);                  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = batch_enqueue(b, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        b->tiles[name] = best;
    }
    if (e == cudaSuccess) e = batch_upload(b);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_batch_run(interp_batch_t *b, void *stream)
{
    if (!b) return INTERP_EINVAL;
    cudaError_t e = cudaSuccess;
    if (b->dirty) {
        batch_free_graph(b);
        e = cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e_enq = batch_enqueue(b, b->cs);
            e = cudaStreamEndCapture(b->cs, &b->graph);
            if (e_enq != cudaSuccess) e = e_enq;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            batch_free_graph(b);
            cudaGetLastError();
            return cuda_status(e);
        }
        b->dirty = false;
    }
    e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

}  // extern "C"

