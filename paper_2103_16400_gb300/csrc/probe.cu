// Measurement support (no counterpart in the paper): throughput probes that
// give the integer roofline its denominator, and the launch counter.
//
// hx_probe_int_mul_rate: every thread runs 8 independent dependency chains of
// one 32-bit integer multiply form (kind 0: mad.lo.u32, the low half of a
// 32x32-bit product plus an addend; kind 1: mad.hi.u32, the high half;
// kind 2: mad.wide.u32, the full 64-bit product; kind 3: lo and hi
// alternating).  The grid fills every SM; the rate is
// (threads x iterations x 16 instructions) / elapsed time.
//
// hx_probe_copy_rate: a 16-byte grid-stride copy between any two addresses
// the GPU can reach (device memory, or pinned host memory through unified
// addressing), timed like the others.
//
// hx_probe_butterfly_rate: the same grid runs Harvey forward or inverse
// butterflies on register-resident data (no memory traffic), giving the
// arithmetic ceiling of each Shoup-product variant of the butterfly code
// (variants 0-2: exact quotient, lazy bound 2q; 3: truncated quotient, 4q).
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "hx_internal.h"
#include "modarith.cuh"

namespace hx {

std::atomic<uint64_t> g_launches{0};

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------- launch timing
// While enabled, the NTT pass launches and the fused tensor pass record a pair
// of CUDA events around themselves on their own stream (timing_begin before
// the launch, timing_end after it).  The events are created when timing is
// enabled and come back to the pool when the records are read.
struct TimedLaunch {
    cudaEvent_t a, b;
    uint32_t kernel;
};
static std::mutex g_tm_mu;
static bool g_tm_on = false;
static uint32_t g_tm_cap = 0;
static uint32_t g_tm_gen = 0;   // bumped by every read: a slot from before a read is void
static std::vector<TimedLaunch> g_tm;
static std::vector<cudaEvent_t> g_tm_pool;

uint32_t timing_begin(cudaStream_t s, uint32_t kernel) {
    std::lock_guard<std::mutex> g(g_tm_mu);
    if (!g_tm_on || g_tm.size() >= g_tm_cap || g_tm_pool.size() < 2) return 0;
    TimedLaunch t;
    t.b = g_tm_pool.back();
    g_tm_pool.pop_back();
    t.a = g_tm_pool.back();
    g_tm_pool.pop_back();
    t.kernel = kernel;
    if (cudaEventRecord(t.a, s) != cudaSuccess) {
        g_tm_pool.push_back(t.a);
        g_tm_pool.push_back(t.b);
        return 0;
    }
    g_tm.push_back(t);
    return ((g_tm_gen & 0x7ffu) << 21) | (uint32_t)g_tm.size();   // generation | index + 1
}

void timing_end(uint32_t slot, cudaStream_t s) {
    if (!slot) return;
    std::lock_guard<std::mutex> g(g_tm_mu);
    const uint32_t idx = slot & ((1u << 21) - 1);
    if ((slot >> 21) == (g_tm_gen & 0x7ffu) && idx <= g_tm.size())
        cudaEventRecord(g_tm[idx - 1].b, s);
}

static const char* kKernelNames[8] = {"ntt_pass_kernel",       "ntt_pipe_kernel",
                                      "ntt_tensor_inv_kernel", "ntt_cluster_kernel",
                                      "ntt_cluster_tensor_kernel", "ntt_mul_inv_kernel",
                                      "ntt_ct_row_kernel",     "ntt_mul_row_kernel"};

template <int KIND>
__global__ void __launch_bounds__(256) int_mul_probe_kernel(uint32_t iters, uint32_t a,
                                                            uint32_t b, uint32_t* sink) {
    uint32_t x[8];
    uint64_t y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        x[i] = threadIdx.x * 7u + i;
        y[i] = x[i];
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (KIND == 0 || (KIND == 3 && h == 0))
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(a), "r"(b));
                else if (KIND == 1 || KIND == 3)
                    asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(a), "r"(b));
                else
                    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(y[i]) : "r"((uint32_t)y[i]), "r"(a));
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i] ^ (uint32_t)y[i] ^ (uint32_t)(y[i] >> 32);
    if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;   // keeps the chains live
}

template <typename Wd, int V, bool INV>
__global__ void __launch_bounds__(256) butterfly_probe_kernel(uint32_t iters, uint64_t q,
                                                              uint64_t w, uint64_t wp,
                                                              uint64_t* sink) {
    Wd x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (Wd)((threadIdx.x * 131u + i) % q);
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            if constexpr (sizeof(Wd) == 8) {
                const uint64_t m = (V == 3 ? 4 : 2) * q;
                if (INV)
                    harvey_inv64<V>(x[i], x[i + 1], w, wp, q, m);
                else
                    harvey_fwd64<V>(x[i], x[i + 1], w, wp, q, m);
            } else {
                if (INV)
                    harvey_inv32(x[i], x[i + 1], (uint32_t)w, (uint32_t)wp, (uint32_t)q,
                                 (uint32_t)(2 * q));
                else
                    harvey_fwd32(x[i], x[i + 1], (uint32_t)w, (uint32_t)wp, (uint32_t)q,
                                 (uint32_t)(2 * q));
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {   // re-pair so the chains mix
            Wd t = x[i];
            x[i] = x[7 - i];
            x[7 - i] = t;
        }
        // an opaque register move per iteration keeps the loop from being folded
        asm volatile("" : "+r"(*(uint32_t*)&x[0]));
    }
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= (uint64_t)x[i];
    if (acc == 0x9e3779b97f4a7c15ull) sink[blockIdx.x] = acc;
}

// 16-byte grid-stride copy; src or dst may be pinned host memory (reached
// over the CPU-GPU link through unified addressing).
__global__ void __launch_bounds__(256) copy16_kernel(uint4* __restrict__ dst,
                                                     const uint4* __restrict__ src, uint64_t n16) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {   // four loads in flight per thread
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride],
                    d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n16; i += stride) dst[i] = src[i];
}

typedef void (*BflyKernel)(uint32_t, uint64_t, uint64_t, uint64_t, uint64_t*);

template <int V>
static BflyKernel bfly_kernel(bool narrow, bool inv) {
    if (narrow) return inv ? butterfly_probe_kernel<uint32_t, V, true>
                           : butterfly_probe_kernel<uint32_t, V, false>;
    return inv ? butterfly_probe_kernel<uint64_t, V, true> : butterfly_probe_kernel<uint64_t, V, false>;
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

typedef void (*ProbeKernel)(uint32_t, uint32_t, uint32_t, uint32_t*);

// Times `launch(iters)` after one short warm-up launch; returns ms or < 0.
template <class F>
static float time_probe(cudaStream_t st, F launch, uint32_t iters) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch(iters / 8 + 1);
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1.f;
    return t;
}

}  // namespace hx

using namespace hx;

extern "C" uint64_t hx_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" int hx_timing_enable(int on, uint32_t capacity) {
    std::lock_guard<std::mutex> g(g_tm_mu);
    if (!on) {
        g_tm_on = false;
        return HX_OK;
    }
    if (capacity == 0 || capacity > (1u << 20)) return HX_ERR_ARG;
    // events for every record not yet read and every one still to come
    const size_t want = 2 * ((size_t)capacity - std::min<size_t>(capacity, g_tm.size()));
    while (g_tm_pool.size() < want) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return HX_ERR_CUDA;
        g_tm_pool.push_back(e);
    }
    g_tm_cap = capacity;
    g_tm_on = true;
    return HX_OK;
}

extern "C" int hx_timing_read(hx_launch_time* h_out, uint32_t cap, uint32_t* n_out) {
    if (!n_out || (!h_out && cap)) return HX_ERR_NULL;
    std::lock_guard<std::mutex> g(g_tm_mu);
    uint32_t n = 0;
    int st = HX_OK;
    for (const TimedLaunch& t : g_tm) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess)
            st = HX_ERR_CUDA;
        else if (n < cap)
            h_out[n++] = hx_launch_time{t.kernel, 0, ms, 0.f};
        g_tm_pool.push_back(t.a);
        g_tm_pool.push_back(t.b);
    }
    g_tm.clear();
    ++g_tm_gen;
    *n_out = n;
    return st;
}

extern "C" int hx_kernel_name(uint32_t kernel, char* buf, uint32_t len) {
    if (!buf || !len) return HX_ERR_NULL;
    const uint32_t kind = kernel & 3u, fwd = (kernel >> 2) & 1u, column = (kernel >> 3) & 1u;
    const uint32_t logR = (kernel >> 4) & 7u, K = (kernel >> 7) & 31u;
    const uint32_t np = (kernel >> 12) & 3u, tws = (kernel >> 14) & 1u;
    int w;
    if (kind == 0 && ((kernel >> 15) & 1u))   // the product-fused inverse first pass
        w = snprintf(buf, len, "%s<%u, %u, %u, %u>", kKernelNames[5], logR, K, np, tws);
    else if (kind == 0)
        w = snprintf(buf, len, "%s<%u, %u, %u, %u, %u, %u>", kKernelNames[0], fwd, column, logR,
                     K, np, tws);
    else if (kind == 1)
        w = snprintf(buf, len, "%s<%u, %u, %u, %u>", kKernelNames[1], fwd, column, logR, K);
    else if (kind == 2 && ((kernel >> 16) & 1u))   // forward rows, tensor or product, inverse rows
        w = snprintf(buf, len, "%s<%u, %u>", kKernelNames[(kernel >> 17) & 1u ? 7 : 6], logR, K);
    else if (kind == 2)
        w = snprintf(buf, len, "%s<%u, %u, %u, %u>", kKernelNames[2], logR, K, tws, np);
    else if ((kernel >> 12) & 1u)   // cluster-fused: K holds K1, bits 15-19 K2
        w = snprintf(buf, len, "%s<%u, %u, %u>", kKernelNames[4], logR, K, (kernel >> 15) & 31u);
    else
        w = snprintf(buf, len, "%s<%u, %u, %u, %u>", kKernelNames[3], fwd, logR, K,
                     (kernel >> 15) & 31u);
    return w < 0 || (uint32_t)w >= len ? HX_ERR_CAPACITY : HX_OK;
}

extern "C" int hx_probe_int_mul_rate(uint32_t kind, uint32_t iters, double* ops_per_s, float* ms,
                                     hx_stream_t stream) {
    if (!ops_per_s) return HX_ERR_NULL;
    if (iters == 0 || kind > 3) return HX_ERR_ARG;
    static const ProbeKernel kernels[4] = {int_mul_probe_kernel<0>, int_mul_probe_kernel<1>,
                                           int_mul_probe_kernel<2>, int_mul_probe_kernel<3>};
    const int blocks = sm_count() * 8;
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, blocks * sizeof(uint32_t)) != cudaSuccess) return HX_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    ProbeKernel k = kernels[kind];
    float t = time_probe(st, [&](uint32_t it) {
        k<<<blocks, 256, 0, st>>>(it, 0x9e3779b1u, 0x7f4a7c15u, sink);
    }, iters);
    cudaFree(sink);
    if (t <= 0) return HX_ERR_CUDA;
    *ops_per_s = (double)blocks * 256.0 * iters * 16.0 / (t * 1e-3);
    if (ms) *ms = t;
    return HX_OK;
}

extern "C" int hx_probe_butterfly_rate(uint32_t variant, uint32_t iters, uint64_t q,
                                       double* butterflies_per_s, float* ms, hx_stream_t stream) {
    if (!butterflies_per_s) return HX_ERR_NULL;
    const uint32_t v = variant & 15u;
    const bool inv = (variant >> 4) & 1u;
    if (iters == 0 || q < 3 || q >= (1ull << 62) || v > 3) return HX_ERR_ARG;
    if (v == 3 && q >= (1ull << 61)) return HX_ERR_ARG;
    const int blocks = sm_count() * 8;
    uint64_t* sink = nullptr;
    if (cudaMalloc(&sink, blocks * sizeof(uint64_t)) != cudaSuccess) return HX_ERR_NOMEM;
    const uint64_t w = q / 3 + 1;
    const bool narrow = q < (1ull << 30);
    const uint64_t wp = narrow ? ((w << 32) / q) : (uint64_t)(((unsigned __int128)w << 64) / q);
    BflyKernel k = v == 0   ? bfly_kernel<0>(narrow, inv)
                   : v == 1 ? bfly_kernel<1>(narrow, inv)
                   : v == 2 ? bfly_kernel<2>(narrow, inv)
                            : bfly_kernel<3>(narrow, inv);
    cudaStream_t st = (cudaStream_t)stream;
    float t = time_probe(st, [&](uint32_t it) { k<<<blocks, 256, 0, st>>>(it, q, w, wp, sink); },
                         iters);
    cudaFree(sink);
    if (t <= 0) return HX_ERR_CUDA;
    *butterflies_per_s = (double)blocks * 256.0 * iters * 4.0 / (t * 1e-3);
    if (ms) *ms = t;
    return HX_OK;
}

extern "C" int hx_probe_copy_rate(void* dst, const void* src, uint64_t bytes, uint32_t iters,
                                  uint32_t blocks_per_sm, double* bytes_per_s, float* ms,
                                  hx_stream_t stream) {
    if (!dst || !src || !bytes_per_s) return HX_ERR_NULL;
    if (bytes == 0 || (bytes & 15) || ((uintptr_t)dst & 15) || ((uintptr_t)src & 15) ||
        iters == 0 || blocks_per_sm == 0 || blocks_per_sm > 32)
        return HX_ERR_ARG;
    // only device memory or registered (pinned) host memory, through the
    // device-side address the runtime reports for it
    void* ends[2] = {dst, const_cast<void*>(src)};
    for (auto& p : ends) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return HX_ERR_ARG;
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeHost &&
            at.type != cudaMemoryTypeManaged)
            return HX_ERR_ARG;
        if (!at.devicePointer) return HX_ERR_ARG;
        p = at.devicePointer;
    }
    const int blocks = sm_count() * (int)blocks_per_sm;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t n16 = bytes / 16;
    uint4* d = (uint4*)ends[0];
    const uint4* sr = (const uint4*)ends[1];
    float t = time_probe(st, [&](uint32_t it) {
        for (uint32_t k = 0; k < it; ++k) copy16_kernel<<<blocks, 256, 0, st>>>(d, sr, n16);
    }, iters);
    if (t <= 0) return HX_ERR_CUDA;
    *bytes_per_s = (double)bytes * iters / (t * 1e-3);
    if (ms) *ms = t / iters;
    return HX_OK;
}
