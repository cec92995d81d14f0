// peaks.cu -- microbenchmarks of the B300 resources the evaluator's kernels are bound by.
//
// The rooflines of the evaluator divide by these measured rates, not by spec-sheet products:
//   * FP32 FMA throughput (the bound of ray-coherent and spatially sorted queries, whose
//     coefficient gathers hit L1);
//   * L2-resident read bandwidth (coalesced 16-byte loads over a buffer that fits L2);
//   * random gather rates: loads of 4, 16 or 32 bytes at pseudo-random addresses, each inside
//     one 32-byte sector, from an L2-resident buffer (every load its own L1 miss and L1 -> L2
//     request: the access pattern of the coefficient gathers of random queries) and from an
//     L1-resident one (every load a hit: the L1 lookup rate of divergent loads);
//   * L2 atomic throughput: red.global.add.f32 at pseudo-random addresses of an L2-resident
//     buffer (the scatter of the adjoint);
//   * shared-memory atomic throughput, float and integer add at pseudo-random words (the
//     binned adjoint sums its contributions with shared-memory float atomics).
// Each entry point launches one kernel on the caller's stream; the caller times it with CUDA
// events and converts with the work counts documented beside each entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace {

// FMA chains: NCH independent accumulators per thread, ITER rounds of NCH FMAs each
constexpr int kFmaChains = 8;
constexpr int kFmaUnroll = 64;

__global__ void __launch_bounds__(256) k_fma(float *out, int iters, float a, float b)
{
    float acc[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) acc[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kFmaUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kFmaChains; ++c) acc[c] = fmaf(acc[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += acc[c];
    // never true for the arguments the runner passes; keeps the chains live
    if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// coalesced float4 reads of an L2-resident buffer, `passes` times over
__global__ void __launch_bounds__(256) k_l2_read(const float4 *__restrict__ buf, int64_t n4, int passes,
                                                 float *__restrict__ out)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// pseudo-random word index in [0, mask]: one multiply-add per step of a 32-bit LCG
__device__ __forceinline__ uint32_t lcg(uint32_t x) { return x * 1664525u + 1013904223u; }

// one W-float load at element offset i of buf (W = 1, 4 or 8; 8 is one 32-byte sector)
template <int W>
__device__ __forceinline__ float load_w(const float *__restrict__ buf, uint32_t i)
{
    if constexpr (W == 1) {
        return __ldg(buf + i);
    } else if constexpr (W == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(buf) + i);
        return (v.x + v.y) + (v.z + v.w);
    } else {
        float a[8];
        asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7])
                     : "l"(buf + 8 * (size_t)i));
        return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
}

// each thread: `iters` rounds of 8 independent W-float loads at pseudo-random W-aligned addresses
// (each inside one 32-byte sector); the buffer holds mask + 1 W-vectors (a power of two)
template <int W>
__global__ void __launch_bounds__(128) k_gather(const float *__restrict__ buf, uint32_t mask, int iters,
                                                float *__restrict__ out)
{
    uint32_t st[8];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int u = 0; u < 8; ++u) st[u] = lcg(t * 8u + (uint32_t)u + 0x9e3779b9u);
    float acc = 0.0f;
    for (int i = 0; i < iters; ++i) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            st[u] = lcg(st[u]);
            v[u] = load_w<W>(buf, (st[u] >> 4) & mask);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    if (acc == 1234.5f) out[t] = acc;
}

// groups of G lanes (adjacent lanes of one warp) share a pseudo-random 128-byte line: in every
// load instruction lane r of a group reads the word at float offset r * (32 / G) of its group's
// line, so one instruction asks for G different sectors of each of 32 / G lines (the buffer holds
// mask + 1 lines of 32 floats; mask + 1 a power of two)
template <int G>
__global__ void __launch_bounds__(128) k_gather_lines(const float *__restrict__ buf, uint32_t mask, int iters,
                                                      float *__restrict__ out)
{
    uint32_t st[8];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t grp = t / G, r = t % G;
#pragma unroll
    for (int u = 0; u < 8; ++u) st[u] = lcg(grp * 8u + (uint32_t)u + 0x9e3779b9u);
    float acc = 0.0f;
    for (int i = 0; i < iters; ++i) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            st[u] = lcg(st[u]);
            v[u] = __ldg(buf + 32 * (size_t)((st[u] >> 4) & mask) + r * (32 / G));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    if (acc == 1234.5f) out[t] = acc;
}

// ---- tensor cores: tcgen05.mma kind::tf32, D[128 x 128] (+)= A[128 x 32] B[128 x 32]^T per CTA
// Both operands K-major in shared memory with the 128-byte swizzle (16-byte chunk c of row r at
// chunk c ^ (r mod 8), 8-row groups 1024 bytes apart), the accumulator in TMEM (128 lanes x 128
// FP32 columns), completion tracked by an mbarrier with a bounded wait (err = 1 on time-out).
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);            // start address / 16
    d |= (uint64_t)1 << 16;                             // leading byte offset (unused: K fits one row)
    d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;        // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                             // descriptor version
    d |= (uint64_t)2 << 61;                             // 128-byte swizzle
    return d;
}

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M x N
constexpr uint32_t tc_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// every CTA: iters x 4 MMAs of 128 x 128 x 8 accumulating one 128 x 128 x 32 product per
// iteration; CTA 0 writes its accumulator to D (iters = 1: D = A B^T)
__global__ void __launch_bounds__(128) k_tc_tf32(const float *__restrict__ A, const float *__restrict__ B,
                                                 float *__restrict__ D, int iters, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    unsigned char *base = (unsigned char *)(((uintptr_t)tc_sm + 1023) & ~(uintptr_t)1023);
    float *sA = (float *)base;
    float *sB = (float *)(base + 16384);
    uint64_t *mbar = (uint64_t *)(base + 32768);
    uint32_t *taddr_s = (uint32_t *)(base + 32768 + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 128 * 32; i += 128) {
        const int row = i >> 5, k = i & 31;
        const int p = row * 32 + (((k >> 2) ^ (row & 7)) << 2) + (k & 3);
        sA[p] = A[i];
        sB[p] = B[i];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(taddr_s)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *taddr_s;
    if (tid == 0) {
        const uint32_t id = tc_idesc_tf32(128, 128);
        for (int it = 0; it < iters; ++it) {
            for (int k = 0; k < 4; ++k) {
                const uint64_t da = tc_desc_sw128(smem_u32(sA) + k * 32);
                const uint64_t db = tc_desc_sw128(smem_u32(sB) + k * 32);
                const uint32_t acc = (it | k) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                             ::"r"(taddr), "l"(da), "l"(db), "r"(id), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
    }
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(mbar)));
    done = __all_sync(0xffffffffu, done);
    if (!done && lane == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (done && blockIdx.x == 0) {
        for (int half = 0; half < 2; ++half) {
            uint32_t r[32];
            for (int q = 0; q < 2; ++q) {
                const uint32_t a = taddr + ((uint32_t)(warp * 32) << 16) + half * 64 + q * 32;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                             "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                               "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                               "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                               "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                             : "r"(a));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                for (int j = 0; j < 32; ++j) D[(warp * 32 + lane) * 128 + half * 64 + q * 32 + j] = __uint_as_float(r[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(taddr));
}

// each thread: `iters` rounds of 4 red.global.add.f32 at pseudo-random word addresses
__global__ void __launch_bounds__(128) k_red(float *__restrict__ buf, uint32_t mask, int iters)
{
    uint32_t st[4];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) st[u] = lcg(t * 4u + (uint32_t)u + 0x7f4a7c15u);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            st[u] = lcg(st[u]);
            atomicAdd(buf + ((st[u] >> 4) & mask), 1.0f);
        }
    }
}

// shared-memory atomics: 8 per thread and round at pseudo-random elements of a 4096-element
// block-local array: float add (T = 0), 32-bit integer add (T = 1), 64-bit integer add (T = 2)
// T = 3: a 64-bit fixed-point sum kept as two 32-bit words: the low word by an integer add that
// returns the old value, the high word only when the value's high part plus the carry is not
// zero (values +-0.75 scaled by 2^40, alternating in sign)
__global__ void __launch_bounds__(256) k_shared_fixed(int iters, float *__restrict__ out)
{
    __shared__ unsigned slo[4096];
    __shared__ int shi[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) {
        slo[i] = 0u;
        shi[i] = 0;
    }
    __syncthreads();
    uint32_t st = lcg(blockIdx.x * blockDim.x + threadIdx.x);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            st = lcg(st);
            const float v = (st & 256u) ? -0.75f : 0.75f;
            const long long q = __float2ll_rn(v * 0x1p40f);
            const unsigned lo = (unsigned)q;
            const unsigned e = (st >> 8) & 4095u;
            const unsigned old = atomicAdd(&slo[e], lo);
            const int hi = (int)(q >> 32) + (old + lo < old ? 1 : 0);
            if (hi != 0) atomicAdd(&shi[e], hi);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) out[blockIdx.x] = (float)slo[0] + (float)shi[0];
}

template <int T>
__global__ void __launch_bounds__(256) k_shared_atomic(int iters, float *__restrict__ out)
{
    using E = std::conditional_t<T == 0, float, std::conditional_t<T == 1, unsigned, unsigned long long>>;
    __shared__ E sa[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) sa[i] = E(0);
    __syncthreads();
    uint32_t st = lcg(blockIdx.x * blockDim.x + threadIdx.x);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            st = lcg(st);
            atomicAdd(&sa[(st >> 8) & 4095u], E(1));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) out[blockIdx.x] = (float)sa[threadIdx.x];
}

}  // namespace

extern "C" {

// FP32 FMA: grid x 256 threads, each 8 chains x 64 x iters FMAs (2 FLOP each).
// FLOP = grid * 256 * 8 * 64 * iters * 2.  `out` (grid * 256 floats) is never written.
int peaks_fma(int grid, int iters, float *out, void *stream)
{
    k_fma<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, 0.999999f, 1e-7f);
    return (int)cudaPeekAtLastError();
}

// L2-resident read: bytes = n4 * 16 * passes.  `out` (grid * 256 floats) is never written.
int peaks_l2_read(const void *buf, int64_t n4, int passes, int grid, float *out, void *stream)
{
    k_l2_read<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const float4 *>(buf), n4, passes,
                                                                     out);
    return (int)cudaPeekAtLastError();
}

// random gather: loads = grid * 128 * 8 * iters, each of `width` floats (1, 4 or 8) inside one
// 32-byte sector; buf holds (mask + 1) * width floats (mask + 1 a power of two) and is 32-byte
// aligned.  `out` (grid * 128 floats) is never written.
int peaks_gather(const float *buf, uint32_t mask, int width, int grid, int iters, float *out, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (width == 1) k_gather<1><<<grid, 128, 0, st>>>(buf, mask, iters, out);
    else if (width == 4) k_gather<4><<<grid, 128, 0, st>>>(buf, mask, iters, out);
    else if (width == 8) k_gather<8><<<grid, 128, 0, st>>>(buf, mask, iters, out);
    else return (int)cudaErrorInvalidValue;
    return (int)cudaPeekAtLastError();
}

// random line gathers: grid * 128 * 8 * iters loads, groups of `group` (1, 2 or 4) lanes on one
// line; buf holds mask + 1 lines of 128 bytes
int peaks_gather_lines(const float *buf, uint32_t mask, int group, int grid, int iters, float *out, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (group == 1) k_gather_lines<1><<<grid, 128, 0, st>>>(buf, mask, iters, out);
    else if (group == 2) k_gather_lines<2><<<grid, 128, 0, st>>>(buf, mask, iters, out);
    else if (group == 4) k_gather_lines<4><<<grid, 128, 0, st>>>(buf, mask, iters, out);
    else return (int)cudaErrorInvalidValue;
    return (int)cudaPeekAtLastError();
}

// tensor-core TF32 products: grid CTAs x iters x 2 x 128 x 128 x 32 FLOP; D (128 x 128) from CTA
// 0; A, B: 128 x 32 row-major; err (one int, zeroed by the caller) set on a time-out
int peaks_tc_tf32(const float *A, const float *B, float *D, int grid, int iters, int *err, void *stream)
{
    const int smem = 32768 + 1024 + 64;
    cudaError_t e = cudaFuncSetAttribute(k_tc_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    k_tc_tf32<<<grid, 128, smem, static_cast<cudaStream_t>(stream)>>>(A, B, D, iters, err);
    return (int)cudaPeekAtLastError();
}

// random L2 atomics: red.add.f32 count = grid * 128 * 4 * iters into buf (mask + 1 floats)
int peaks_red(float *buf, uint32_t mask, int grid, int iters, void *stream)
{
    k_red<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(buf, mask, iters);
    return (int)cudaPeekAtLastError();
}

// shared-memory atomics: count = grid * 256 * 8 * iters; type 0 float add, 1 32-bit integer add,
// 2 64-bit integer add, 3 64-bit fixed-point add as two 32-bit words.  `out`
// (grid floats) receives one value per CTA.
int peaks_shared_atomic(int type, int grid, int iters, float *out, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (type == 0) k_shared_atomic<0><<<grid, 256, 0, st>>>(iters, out);
    else if (type == 1) k_shared_atomic<1><<<grid, 256, 0, st>>>(iters, out);
    else if (type == 2) k_shared_atomic<2><<<grid, 256, 0, st>>>(iters, out);
    else if (type == 3) k_shared_fixed<<<grid, 256, 0, st>>>(iters, out);
    else return (int)cudaErrorInvalidValue;
    return (int)cudaPeekAtLastError();
}

}  // extern "C"
