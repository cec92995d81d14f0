// interp.cu -- C ABI of the lattice convolution-sum evaluator (see include/interp.h).
//
// Host side: handle creation (matching (L, Xi) against the generated splines), halo-padded
// coefficient storage, conversion of user coefficients, and launches of the kernels in
// kernels.cuh on the caller's stream.  No host computation of results, no fallback path.
#include "interp.h"

#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <type_traits>

#include "generated/splines.h"

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
};

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
        if (o.s != s || o.nxi != n || o.D != li.D || o.M != (int)li.cosets.size()) continue;
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
    if (!ibl::make_layout(h->lay, s, h->dims, pad, esz, ops->M) ||
        !ibl::make_layout(h->lay32, s, h->dims, pad, 4, ops->M)) {
        delete h;
        return INTERP_ESIZE;
    }
    h->coeff_count = cc * ops->M;
    cudaGetDevice(&h->device);
    const size_t bytes = (size_t)h->lay.coset_elems * ops->M * esz;
    cudaError_t e = cudaMalloc(&h->coeffs, bytes);
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

void interp_destroy(interp_t *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->coeffs);
    cudaFree(h->dpad);
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
    return INTERP_OK;
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
        e = cudaMallocAsync(&tmp, bytes, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            if (tmp) cudaFreeAsync(tmp, st);
            cudaGetLastError();
            return cuda_status(e);
        }
        dsrc = tmp;
    }
    const unsigned grid = (unsigned)std::min<int64_t>((h->coeff_count + 255) / 256, 148 * 32);
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
    const int dt = h->storage == INTERP_F32 ? 0 : (h->storage == INTERP_F16 ? 1 : 2);
    cudaError_t e = h->ops->eval[dt][mode](pts, npts, h->coeffs, h->lay, out, grad, gout,
                                           static_cast<cudaStream_t>(stream));
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
    const size_t dbytes = (size_t)h->lay32.coset_elems * h->ops->M * sizeof(float);
    if (!h->dpad) {
        e = cudaMalloc(&h->dpad, dbytes);
        if (e != cudaSuccess) {
            h->dpad = nullptr;
            cudaGetLastError();
            return cuda_status(e);
        }
    }
    e = cudaMemsetAsync(h->dpad, 0, dbytes, st);
    if (e == cudaSuccess) e = h->ops->adjoint(pts, npts, gout, h->lay32, h->dpad, st);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::min<int64_t>((h->coeff_count + 255) / 256, 148 * 32);
        k_unpad_add<<<grid, 256, 0, st>>>(h->dpad, dcoeffs, h->coeff_count, h->lay32);
        e = cudaPeekAtLastError();
    }
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

interp_status interp_backward_noalloc(interp_t *h, const float *pts, int64_t npts, const float *gout, float *dcoeffs,
                                      float *dpts, void *stream)
{
    if (!h || npts < 0) return INTERP_EINVAL;
    const int64_t need = (int64_t)h->lay32.coset_elems * h->ops->M;
    if (need > INTERP_NOALLOC_MAX_GRAD_ELEMS) return INTERP_ESIZE;
    if (npts == 0) return INTERP_OK;
    if (!pts || !gout) return INTERP_EINVAL;
    if (npts > (int64_t)INT32_MAX * kTPB) return INTERP_ESIZE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return INTERP_ECUDA;
    }
    if (dev != h->device) return INTERP_EINVAL;
    if (dpts) {
        interp_status s2 = eval_common(h, pts, npts, nullptr, dpts, gout, 2, stream);
        if (s2 != INTERP_OK) return s2;
    }
    if (!dcoeffs) return INTERP_OK;
    float *scratch = nullptr;
    interp_status st0 = noalloc_scratch(dev, &scratch);
    if (st0 != INTERP_OK) return st0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(scratch, 0, (size_t)need * sizeof(float), st);
    if (e == cudaSuccess) e = h->ops->adjoint(pts, npts, gout, h->lay32, scratch, st);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::min<int64_t>((h->coeff_count + 255) / 256, 148 * 32);
        k_unpad_add<<<grid, 256, 0, st>>>(scratch, dcoeffs, h->coeff_count, h->lay32);
        e = cudaPeekAtLastError();
    }
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
