// Ragged batches: many transforms of different N (2^10 .. 2^17) and different
// modulus sets run as one persistent kernel per pass, replayed as one CUDA
// graph.
//
// Every transform is cut into tiles of 2048 elements (1024 at N = 2^10), in
// pass shapes chosen per log2 N from a menu:
//   N = 2^10, 2^11      one pass over all stages (S10, S11)
//   N = 2^12 .. 2^17    a column pass over the first K1 stages (C5..C9) and a
//                       row pass over the last K2 (R6..R11), K1 + K2 = log2 N;
//                       the split K1 per log2 N is a process-wide setting
//                       (hx_ragged_set_split) that the autotuner chooses
// The host writes one 32-byte descriptor per tile (operand and result
// pointers, the limb's constants, tile index, menu entry); a persistent grid of
// 256-thread blocks takes tiles from the list through an atomic counter, so
// blocks that draw small or narrow tiles simply take more of them.  The
// second pass of two-pass transforms is a second launch of the same kernel
// over its own list.  The counters are the batch's only scratch memory; a
// memset node re-arms them at the head of the graph on every replay.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "ntt_kernels.cuh"

namespace hx {

struct RagTile {
    const uint64_t* in;   // this transform's operand, element 0
    uint64_t* out;        // this transform's result, element 0
    const LimbDev* lc;    // its limb constants (twiddle tables inside)
    uint32_t tile;        // tile index within the pass
    uint8_t kind;         // menu entry
    uint8_t L;            // log2 N
    uint8_t last;         // this pass finishes the transform
    uint8_t out_mf;
};
static_assert(sizeof(RagTile) == 32, "descriptor is 32 bytes");

enum RagKind : uint8_t {
    RK_S10 = 0, RK_S11, RK_C5, RK_C6, RK_C7, RK_C8, RK_R7, RK_R8, RK_R9,
    RK_C9, RK_R6, RK_R10, RK_R11
};

static int col_kind(int K1) { return K1 == 9 ? RK_C9 : RK_C5 + (K1 - 5); }
static int row_kind(int K2) {
    return K2 == 6 ? RK_R6 : K2 <= 9 ? RK_R7 + (K2 - 7) : K2 == 10 ? RK_R10 : RK_R11;
}

// The column-pass stage count K1 per log2 N (the row pass takes the other
// log2 N - K1), process-wide; the defaults are the shapes measured best on
// GB300 before the tuner existed.
static std::atomic<int> g_rag_split[18] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,
                                           5, 6, 7, 7, 8, 8};

// A split is in the menu when both passes fit a 2048-element tile of 256
// threads: column passes of 5 .. 9 stages (2^(11-K1) >= 4 columns), row
// passes of 6 .. 11.
static bool split_ok(int L, int K1) {
    return L >= 12 && L <= 17 && K1 >= 5 && K1 <= 9 && L - K1 >= 6 && L - K1 <= 11;
}

// kinds of the first (column or single) and second (row) pass for log2 N
static void rag_kinds(int L, int* first, int* second) {
    if (L == 10 || L == 11) {
        *first = L == 10 ? RK_S10 : RK_S11;
        *second = -1;
        return;
    }
    const int K1 = g_rag_split[L].load(std::memory_order_relaxed);
    *first = col_kind(K1);
    *second = row_kind(L - K1);
}

// One tile: geometry from the menu, then the same per-tile code as the plain
// pass kernel.  Tiles hold 2^11 elements (2^10 for S10) in 256 threads.
template <bool FWD, bool COLUMN, int LOG_R, int K>
__device__ __forceinline__ void rag_tile(uint64_t* sm, const RagTile& d) {
    const int L = d.L;
    const int s0 = COLUMN || K >= L ? 0 : L - K;
    const int w = L - s0 - K;
    const int logGc = COLUMN ? 11 - K : 0;
    const int logGb = COLUMN ? 0 : (K >= L ? 0 : 11 - K);
    const int logTE = logGb + K + logGc;
    const int log_tiles_c = w - logGc;
    TileCtx c;
    c.gin = d.in;
    c.gout = d.out;
    c.b_base = (uint64_t)(d.tile >> log_tiles_c) << logGb;
    c.c_base = (uint64_t)(d.tile & ((1u << log_tiles_c) - 1)) << logGc;
    c.L = L;
    c.s0 = s0;
    c.logGc = logGc;
    c.logGb = logGb;
    c.w = w;
    c.nthreads = (1u << logTE) >> LOG_R;
    c.out_mf = d.out_mf;
    c.last = d.last != 0;
    const LimbDev lc = *d.lc;
    process_tile<FWD, COLUMN, LOG_R, K>(sm, c, lc, 1u << logTE);
}

// 64 registers (4 blocks of 256 threads per SM): the kernel holds every menu
// shape behind one switch, and the compiler's own allocation (128, 2 blocks)
// left too few warps to cover the loads -- measured on the 512-polynomial
// ragged batch: 4.92 -> 3.44 ms.
template <bool FWD>
__global__ void __maxnreg__(64) ragged_pass_kernel(const RagTile* __restrict__ tiles,
                                                             uint32_t n, uint32_t* counter) {
    extern __shared__ uint64_t sm[];
    __shared__ uint32_t s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t t = s_next;
        if (t >= n) return;
        const RagTile d = tiles[t];
        switch (d.kind) {
            case RK_S10: rag_tile<FWD, false, 2, 10>(sm, d); break;
            case RK_S11: rag_tile<FWD, false, 3, 11>(sm, d); break;
            case RK_C5: rag_tile<FWD, true, 3, 5>(sm, d); break;
            case RK_C6: rag_tile<FWD, true, 3, 6>(sm, d); break;
            case RK_C7: rag_tile<FWD, true, 3, 7>(sm, d); break;
            case RK_C8: rag_tile<FWD, true, 3, 8>(sm, d); break;
            case RK_C9: rag_tile<FWD, true, 3, 9>(sm, d); break;
            case RK_R6: rag_tile<FWD, false, 3, 6>(sm, d); break;
            case RK_R7: rag_tile<FWD, false, 3, 7>(sm, d); break;
            case RK_R8: rag_tile<FWD, false, 3, 8>(sm, d); break;
            case RK_R10: rag_tile<FWD, false, 3, 10>(sm, d); break;
            case RK_R11: rag_tile<FWD, false, 3, 11>(sm, d); break;
            default: rag_tile<FWD, false, 3, 9>(sm, d); break;
        }
        __syncthreads();   // tile finished with shared memory and s_next
    }
}

static const size_t kRagSmem = padded(2048) * sizeof(uint64_t);

// The inverse's first pass of a ragged product: the tile of a b mod q (both
// spectra from the forward passes, below 4q) computed in the staging step,
// then the row (or single) pass's stages -- the element-wise product never
// goes to HBM.
struct MulRagTile {
    const uint64_t* a;    // this transform's first spectrum, element 0
    const uint64_t* b;    // its second spectrum
    uint64_t* out;        // its result
    const LimbDev* lc;
    uint32_t tile;
    uint8_t kind;         // RK_S10, RK_S11 or a row kind
    uint8_t L;
    uint8_t last;
    uint8_t out_mf;
    uint64_t pad_;
};
static_assert(sizeof(MulRagTile) == 48, "descriptor is 48 bytes");

template <int LOG_R, int K>
__device__ __forceinline__ void rag_mul_tile(uint64_t* sm, const MulRagTile& d) {
    const int L = d.L;
    const int s0 = K >= L ? 0 : L - K;
    const int logGb = K >= L ? 0 : 11 - K;
    const int logTE = logGb + K;
    TileCtx c;
    c.gin = d.a;
    c.gin2 = d.b;
    c.mul_mf = 4;
    c.gout = d.out;
    c.b_base = (uint64_t)d.tile << logGb;
    c.c_base = 0;
    c.L = L;
    c.s0 = s0;
    c.logGc = 0;
    c.logGb = logGb;
    c.w = 0;
    c.nthreads = (1u << logTE) >> LOG_R;
    c.out_mf = d.out_mf;
    c.last = d.last != 0;
    const LimbDev lc = *d.lc;
    process_tile<false, false, LOG_R, K, 1, false, true>(sm, c, lc, 1u << logTE);
}

__global__ void __maxnreg__(64) ragged_mul_inv_kernel(const MulRagTile* __restrict__ tiles,
                                                      uint32_t n, uint32_t* counter) {
    extern __shared__ uint64_t sm[];
    __shared__ uint32_t s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t t = s_next;
        if (t >= n) return;
        const MulRagTile d = tiles[t];
        switch (d.kind) {
            case RK_S10: rag_mul_tile<2, 10>(sm, d); break;
            case RK_S11: rag_mul_tile<3, 11>(sm, d); break;
            case RK_R6: rag_mul_tile<3, 6>(sm, d); break;
            case RK_R7: rag_mul_tile<3, 7>(sm, d); break;
            case RK_R8: rag_mul_tile<3, 8>(sm, d); break;
            case RK_R10: rag_mul_tile<3, 10>(sm, d); break;
            case RK_R11: rag_mul_tile<3, 11>(sm, d); break;
            default: rag_mul_tile<3, 9>(sm, d); break;
        }
        __syncthreads();   // tile finished with shared memory and s_next
    }
}

}  // namespace hx

using namespace hx;

struct hx_batch_s {
    int device = 0;
    bool forward = true;
    uint32_t nA = 0, nB = 0;
    RagTile* d_tiles = nullptr;     // pass A tiles, then pass B tiles
    uint32_t* d_counters = nullptr; // [2]
    int grid = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    uint64_t limb_transforms = 0;
};

static int rag_grid(bool fwd) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (fwd)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ragged_pass_kernel<true>, 256, kRagSmem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ragged_pass_kernel<false>, 256, kRagSmem);
    return std::max(1, per) * std::max(1, sms);
}

static int rag_mul_grid() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ragged_mul_inv_kernel, 256, kRagSmem);
    return std::max(1, per) * std::max(1, sms);
}

// Enqueue one replay of the batch on `st`: re-arm the counters, then the two
// persistent passes.
static cudaError_t rag_enqueue(const hx_batch_s* b, cudaStream_t st, bool capturing) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t ns[2] = {b->nA, b->nB};
    for (int p = 0; p < 2; ++p) {
        if (!ns[p]) continue;
        const RagTile* t = b->d_tiles + (p ? b->nA : 0);
        const unsigned grid = (unsigned)std::min<uint64_t>(ns[p], (uint64_t)b->grid);
        if (b->forward)
            ragged_pass_kernel<true><<<grid, 256, kRagSmem, st>>>(t, ns[p], b->d_counters + p);
        else
            ragged_pass_kernel<false><<<grid, 256, kRagSmem, st>>>(t, ns[p], b->d_counters + p);
        if (!capturing) count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static void rag_free(hx_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_tiles);
    cudaFree(b->d_counters);
    delete b;
}

extern "C" int hx_ragged_set_split(uint32_t log2_n, uint32_t k1) {
    if (!split_ok((int)log2_n, (int)k1)) return HX_ERR_ARG;
    g_rag_split[log2_n].store((int)k1, std::memory_order_relaxed);
    return HX_OK;
}

extern "C" int hx_ragged_get_split(uint32_t log2_n, uint32_t* k1) {
    if (!k1) return HX_ERR_NULL;
    if (log2_n < 12 || log2_n > 17) return HX_ERR_ARG;
    *k1 = (uint32_t)g_rag_split[log2_n].load(std::memory_order_relaxed);
    return HX_OK;
}

extern "C" int hx_batch_create(hx_batch_t* out, const hx_ragged_item* items, uint32_t n_items,
                               uint32_t direction, uint32_t in_mf, uint32_t out_mf) {
    if (!out || !items) return HX_ERR_NULL;
    *out = nullptr;
    if (n_items == 0 || (direction != 1 && direction != 2)) return HX_ERR_ARG;
    const bool fwd = direction == 1;
    if (fwd ? !(in_mf == 1 || in_mf == 2 || in_mf == 4) || !(out_mf == 1 || out_mf == 4)
            : !(in_mf == 1 || in_mf == 2) || !(out_mf == 1 || out_mf == 2))
        return HX_ERR_MOD_FACTOR;
    std::vector<RagTile> A, B;
    uint64_t lt = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    for (uint32_t i = 0; i < n_items; ++i) {
        const hx_ragged_item& it = items[i];
        if (!it.plan || !it.d_in || !it.d_out) return HX_ERR_NULL;
        if (((uintptr_t)it.d_in | (uintptr_t)it.d_out) & 15u) return HX_ERR_ALIGN;
        if (it.n_polys == 0) return HX_ERR_ARG;
        if (it.plan->device != dev) return HX_ERR_ARG;
        const hx_plan_s* p = it.plan;
        const uint64_t bytes = (uint64_t)it.n_polys * p->n_limbs * p->N * 8;
        if (it.d_in != it.d_out && (uintptr_t)it.d_in < (uintptr_t)it.d_out + bytes &&
            (uintptr_t)it.d_out < (uintptr_t)it.d_in + bytes)
            return HX_ERR_OVERLAP;
        int k1, k2;
        rag_kinds(p->logN, &k1, &k2);
        // forward: column/single pass first; inverse: row pass first
        const int first = fwd || k2 < 0 ? k1 : k2, second = k2 < 0 ? -1 : (fwd ? k2 : k1);
        const uint32_t tiles = p->logN <= 11 ? 1u : (1u << (p->logN - 11));
        for (uint32_t poly = 0; poly < it.n_polys; ++poly) {
            for (uint32_t l = 0; l < p->n_limbs; ++l) {
                const uint64_t off = ((uint64_t)poly * p->n_limbs + l) << p->logN;
                for (uint32_t t = 0; t < tiles; ++t) {
                    RagTile a{it.d_in + off, it.d_out + off, p->d_limbs + l, t, (uint8_t)first,
                              (uint8_t)p->logN, (uint8_t)(second < 0), (uint8_t)out_mf};
                    A.push_back(a);
                    if (second >= 0) {
                        RagTile b2{it.d_out + off, it.d_out + off, p->d_limbs + l, t,
                                   (uint8_t)second, (uint8_t)p->logN, 1, (uint8_t)out_mf};
                        B.push_back(b2);
                    }
                }
                ++lt;
            }
        }
    }
    if (A.size() + B.size() >= (1ull << 32)) return HX_ERR_ARG;
    hx_batch_s* b = new (std::nothrow) hx_batch_s();
    if (!b) return HX_ERR_NOMEM;
    b->device = dev;
    b->forward = fwd;
    b->nA = (uint32_t)A.size();
    b->nB = (uint32_t)B.size();
    b->limb_transforms = lt;
    b->grid = rag_grid(fwd);
    if (cudaMalloc((void**)&b->d_tiles, (A.size() + B.size()) * sizeof(RagTile)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_counters, 2 * sizeof(uint32_t)) != cudaSuccess) {
        rag_free(b);
        return HX_ERR_NOMEM;
    }
    if (cudaMemcpy(b->d_tiles, A.data(), A.size() * sizeof(RagTile), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        (B.size() && cudaMemcpy(b->d_tiles + A.size(), B.data(), B.size() * sizeof(RagTile),
                                cudaMemcpyHostToDevice) != cudaSuccess)) {
        rag_free(b);
        return HX_ERR_CUDA;
    }
    // capture one replay into a graph on a private stream
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        rag_free(b);
        return HX_ERR_CUDA;
    }
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = rag_enqueue(b, cs, true);
        cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        rag_free(b);
        return HX_ERR_CUDA;
    }
    *out = b;
    return HX_OK;
}

extern "C" int hx_batch_run(hx_batch_t b, hx_stream_t stream) {
    if (!b) return HX_ERR_NULL;
    if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) return HX_ERR_CUDA;
    count_launch((b->nA ? 1 : 0) + (b->nB ? 1 : 0));
    return HX_OK;
}

extern "C" int hx_batch_info(hx_batch_t b, uint64_t* limb_transforms, uint64_t* tiles,
                             uint32_t* launches) {
    if (!b) return HX_ERR_NULL;
    if (limb_transforms) *limb_transforms = b->limb_transforms;
    if (tiles) *tiles = (uint64_t)b->nA + b->nB;
    if (launches) *launches = (b->nA ? 1 : 0) + (b->nB ? 1 : 0);
    return HX_OK;
}

extern "C" int hx_batch_destroy(hx_batch_t b) {
    if (!b) return HX_ERR_NULL;
    rag_free(b);
    return HX_OK;
}

// ---------------------------------------------------------------------------
// One-shot ragged run for callers that must not allocate device memory.
//
// hx_batch_create allocates its tile list and work counters with cudaMalloc.
// Some callers cannot do that at the point of use: a serving loop that admits
// work against a fixed device-memory budget, an application whose own memory
// pool owns the whole GPU, or a latency-critical path that cannot afford the
// device-wide synchronisation cudaMalloc and cudaFree imply.  For them this
// entry point keeps the counters and the tile list in a fixed array compiled
// into the library (kStaticScratchBytes per GPU that loads it, held until the
// process exits), and calls no cudaMalloc, cudaFree or other allocating
// device routine.
// ---------------------------------------------------------------------------
namespace hx {

constexpr size_t kStaticScratchBytes = 4u << 20;          // 4 MiB per device
constexpr size_t kStaticHeader = 256;                      // the two counters
constexpr uint32_t kStaticMaxTiles =
    (uint32_t)((kStaticScratchBytes - kStaticHeader) / sizeof(RagTile));   // 131064

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The host-side name of g_static_scratch is only a stand-in, not a device
// address; the address is fetched once per device, with that device current.
static std::mutex g_static_mu;
static void* g_static_addr[128];

static int static_scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HX_ERR_CUDA;
    if (dev < 0 || dev >= 128) return HX_ERR_ARG;
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HX_ERR_CUDA;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return HX_OK;
}

}  // namespace hx

namespace hx {

// Checks a ragged set of transforms (the rules of hx_batch_create) and counts
// its tiles: first pass (column or single) and second pass (row).
static int rag_check_count(const hx_ragged_item* items, uint32_t n_items, uint32_t direction,
                           uint32_t in_mf, uint32_t out_mf, uint64_t* n_first,
                           uint64_t* n_second) {
    if (!items) return HX_ERR_NULL;
    if (n_items == 0 || (direction != 1 && direction != 2)) return HX_ERR_ARG;
    const bool fwd = direction == 1;
    if (fwd ? !(in_mf == 1 || in_mf == 2 || in_mf == 4) || !(out_mf == 1 || out_mf == 4)
            : !(in_mf == 1 || in_mf == 2) || !(out_mf == 1 || out_mf == 2))
        return HX_ERR_MOD_FACTOR;
    int dev = 0;
    cudaGetDevice(&dev);
    *n_first = *n_second = 0;
    for (uint32_t i = 0; i < n_items; ++i) {
        const hx_ragged_item& it = items[i];
        if (!it.plan || !it.d_in || !it.d_out) return HX_ERR_NULL;
        if (((uintptr_t)it.d_in | (uintptr_t)it.d_out) & 15u) return HX_ERR_ALIGN;
        if (it.n_polys == 0 || it.plan->device != dev) return HX_ERR_ARG;
        const hx_plan_s* p = it.plan;
        const uint64_t bytes = (uint64_t)it.n_polys * p->n_limbs * p->N * 8;
        if (it.d_in != it.d_out && (uintptr_t)it.d_in < (uintptr_t)it.d_out + bytes &&
            (uintptr_t)it.d_out < (uintptr_t)it.d_in + bytes)
            return HX_ERR_OVERLAP;
        const uint64_t tiles = p->logN <= 11 ? 1u : (1u << (p->logN - 11));
        const uint64_t t = tiles * it.n_polys * p->n_limbs;
        *n_first += t;
        if (p->logN > 11) *n_second += t;
    }
    return HX_OK;
}

// Writes the tile list of a checked set: the n_first first-pass tiles, then
// the n_second second-pass tiles.
static void rag_fill(const hx_ragged_item* items, uint32_t n_items, bool fwd, uint32_t out_mf,
                     RagTile* dst) {
    uint64_t n = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (uint32_t i = 0; i < n_items; ++i) {
            const hx_ragged_item& it = items[i];
            const hx_plan_s* p = it.plan;
            int k1, k2;
            rag_kinds(p->logN, &k1, &k2);
            if (pass == 1 && k2 < 0) continue;
            const int first = fwd || k2 < 0 ? k1 : k2, second = fwd ? k2 : k1;
            const uint32_t nt = p->logN <= 11 ? 1u : (1u << (p->logN - 11));
            for (uint32_t poly = 0; poly < it.n_polys; ++poly) {
                for (uint32_t l = 0; l < p->n_limbs; ++l) {
                    const uint64_t off = ((uint64_t)poly * p->n_limbs + l) << p->logN;
                    for (uint32_t t = 0; t < nt; ++t) {
                        if (pass == 0)
                            dst[n++] = RagTile{it.d_in + off, it.d_out + off, p->d_limbs + l, t,
                                               (uint8_t)first, (uint8_t)p->logN,
                                               (uint8_t)(k2 < 0), (uint8_t)out_mf};
                        else
                            dst[n++] = RagTile{it.d_out + off, it.d_out + off, p->d_limbs + l, t,
                                               (uint8_t)second, (uint8_t)p->logN, 1,
                                               (uint8_t)out_mf};
                    }
                }
            }
        }
    }
}

// Enqueues the two persistent passes over a tile list already on the device.
static int rag_launch(bool fwd, const RagTile* d_tiles, uint64_t n_first, uint64_t n_second,
                      uint32_t* counters, cudaStream_t s) {
    const int grid = rag_grid(fwd);
    const uint64_t ns[2] = {n_first, n_second};
    for (int p = 0; p < 2; ++p) {
        if (!ns[p]) continue;
        const RagTile* t = d_tiles + (p ? n_first : 0);
        const unsigned g = (unsigned)std::min<uint64_t>(ns[p], (uint64_t)grid);
        if (fwd)
            ragged_pass_kernel<true><<<g, 256, kRagSmem, s>>>(t, (uint32_t)ns[p], counters + p);
        else
            ragged_pass_kernel<false><<<g, 256, kRagSmem, s>>>(t, (uint32_t)ns[p], counters + p);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) return HX_ERR_CUDA;
    }
    return HX_OK;
}

}  // namespace hx

extern "C" int hx_batch_run_static(const hx_ragged_item* items, uint32_t n_items,
                                   uint32_t direction, uint32_t in_mf, uint32_t out_mf,
                                   hx_stream_t stream) {
    // count the tiles first, so an oversized request is refused before any work
    uint64_t n_first = 0, n_second = 0;
    int st = rag_check_count(items, n_items, direction, in_mf, out_mf, &n_first, &n_second);
    if (st != HX_OK) return st;
    if (n_first + n_second > kStaticMaxTiles) return HX_ERR_CAPACITY;
    const bool fwd = direction == 1;
    std::vector<RagTile> tiles(n_first + n_second);   // host staging of the tile list
    rag_fill(items, n_items, fwd, out_mf, tiles.data());
    void* base = nullptr;
    st = static_scratch_address(&base);
    if (st != HX_OK) return st;
    uint32_t* counters = (uint32_t*)base;
    RagTile* d_tiles = (RagTile*)((unsigned char*)base + kStaticHeader);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: re-zero the counters
    if (cudaMemsetAsync(counters, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return HX_ERR_CUDA;
    if (cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(RagTile),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return HX_ERR_CUDA;
    return rag_launch(fwd, d_tiles, n_first, n_second, counters, s);
}

// ---------------------------------------------------------------------------
// Ragged polynomial products in a caller-provided workspace (the serving
// primitive).  For every item, c = a * b in R_q per the paper's Listing 4:
// forward NTTs of a and b written out of place into the workspace (outputs
// in [0, 4q)), the element-wise product with input_mod_factor 4, and the
// inverse NTT written straight into the result.  The product runs inside the
// inverse's first pass (its staging step reads both spectra).  Items may
// differ in N and moduli; the whole set is four kernel launches (two forward
// passes, two inverse passes).  The workspace holds the spectra, the tile
// lists and the work counters, so the library allocates nothing.
// ---------------------------------------------------------------------------
namespace hx {

struct PolymulLayout {
    uint64_t spectra = 0;      // bytes of A and B slots
    uint64_t fA = 0, fB = 0, iA = 0, iB = 0;   // descriptor counts (iA: MulRagTile)
    uint64_t tiles_off = 0, total = 0;
};

static int polymul_layout(const hx_polymul_item* items, uint32_t n, PolymulLayout* L) {
    *L = PolymulLayout();
    int dev = 0;
    cudaGetDevice(&dev);
    for (uint32_t i = 0; i < n; ++i) {
        const hx_polymul_item& it = items[i];
        if (!it.plan || !it.d_a || !it.d_b || !it.d_result) return HX_ERR_NULL;
        if (((uintptr_t)it.d_a | (uintptr_t)it.d_b | (uintptr_t)it.d_result) & 15u)
            return HX_ERR_ALIGN;
        if (it.n_polys == 0 || it.plan->device != dev) return HX_ERR_ARG;
        const hx_plan_s* p = it.plan;
        for (uint64_t q : p->moduli)
            if (q >= (1ull << 61)) return HX_ERR_MODULUS;     // 4q < 2^63 for the product
        const uint64_t transforms = (uint64_t)it.n_polys * p->n_limbs;
        const uint64_t tiles = p->logN <= 11 ? 1u : (1u << (p->logN - 11));
        L->spectra += 2 * transforms * p->N * 8;
        L->fA += 2 * transforms * tiles;
        L->iA += transforms * tiles;
        if (p->logN > 11) {
            L->fB += 2 * transforms * tiles;
            L->iB += transforms * tiles;
        }
    }
    L->tiles_off = 256 + L->spectra;
    L->total = L->tiles_off + (L->fA + L->fB + L->iB) * sizeof(RagTile) +
               L->iA * sizeof(MulRagTile);
    if (L->fA + L->fB >= (1ull << 32) || L->iA + L->iB >= (1ull << 32)) return HX_ERR_ARG;
    return HX_OK;
}

}  // namespace hx

extern "C" int hx_polymul_ragged_workspace(const hx_polymul_item* items, uint32_t n_items,
                                           uint64_t* bytes) {
    if (!items || !bytes) return HX_ERR_NULL;
    if (n_items == 0) return HX_ERR_ARG;
    PolymulLayout L;
    int st = polymul_layout(items, n_items, &L);
    if (st != HX_OK) return st;
    *bytes = L.total;
    return HX_OK;
}

// Page-locked host staging for the descriptor lists of hx_polymul_ragged.  A
// copy from pageable memory would first wait for the stream's earlier work and
// then pass through the driver's own staging buffers; from page-locked memory
// it is one asynchronous DMA.  A buffer is handed out again only once the
// event recorded after the copy that last read it has completed; buffers grow
// to the largest list seen and live as long as the process.
struct DescStaging {
    unsigned char* buf = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    int device = -1;
    bool busy = false;
};
static std::mutex g_stage_mu;
static std::vector<DescStaging*> g_stage;

static DescStaging* staging_acquire(size_t bytes, int dev) {
    std::lock_guard<std::mutex> g(g_stage_mu);
    DescStaging* pick = nullptr;
    for (DescStaging* st : g_stage) {
        if (st->device != dev || st->busy) continue;
        if (cudaEventQuery(st->done) != cudaSuccess) continue;   // its copy is in flight
        if (!pick || (st->cap >= bytes && (pick->cap < bytes || st->cap < pick->cap))) pick = st;
    }
    if (!pick) {
        pick = new (std::nothrow) DescStaging();
        if (!pick) return nullptr;
        if (cudaEventCreateWithFlags(&pick->done, cudaEventDisableTiming) != cudaSuccess) {
            delete pick;
            return nullptr;
        }
        pick->device = dev;
        g_stage.push_back(pick);
    }
    if (pick->cap < bytes) {
        size_t cap = 1 << 16;
        while (cap < bytes) cap <<= 1;
        if (pick->buf) cudaFreeHost(pick->buf);
        pick->buf = nullptr;
        pick->cap = 0;
        if (cudaHostAlloc((void**)&pick->buf, cap, cudaHostAllocDefault) != cudaSuccess) {
            pick->buf = nullptr;
            return nullptr;
        }
        pick->cap = cap;
    }
    pick->busy = true;
    return pick;
}

static void staging_release(DescStaging* st) {
    std::lock_guard<std::mutex> g(g_stage_mu);
    st->busy = false;
}

extern "C" int hx_polymul_ragged(const hx_polymul_item* items, uint32_t n_items, void* d_workspace,
                                 uint64_t workspace_bytes, hx_stream_t stream) {
    if (!items || !d_workspace) return HX_ERR_NULL;
    if (n_items == 0) return HX_ERR_ARG;
    if ((uintptr_t)d_workspace & 255u) return HX_ERR_ALIGN;
    PolymulLayout L;
    int st = polymul_layout(items, n_items, &L);
    if (st != HX_OK) return st;
    if (workspace_bytes < L.total) return HX_ERR_CAPACITY;
    unsigned char* ws = (unsigned char*)d_workspace;
    uint32_t* counters = (uint32_t*)ws;
    // descriptors, in launch order: fwd A, fwd B, inv B, then the product-
    // fused first inverse pass (48-byte descriptors, kept last for alignment)
    const size_t host_bytes =
        (L.fA + L.fB + L.iB) * sizeof(RagTile) + L.iA * sizeof(MulRagTile);
    int dev = 0;
    cudaGetDevice(&dev);
    DescStaging* stage = staging_acquire(host_bytes, dev);
    if (!stage) return HX_ERR_NOMEM;
    RagTile* fA = (RagTile*)stage->buf;
    RagTile* fB = fA + L.fA;
    RagTile* iB = fB + L.fB;
    MulRagTile* iA = (MulRagTile*)(iB + L.iB);
    uint64_t nfA = 0, nfB = 0, niA = 0, niB = 0;
    uint64_t* spec = (uint64_t*)(ws + 256);
    for (uint32_t i = 0; i < n_items; ++i) {
        const hx_polymul_item& it = items[i];
        const hx_plan_s* p = it.plan;
        int k1, k2;
        rag_kinds(p->logN, &k1, &k2);
        const uint64_t words = (uint64_t)it.n_polys * p->n_limbs << p->logN;
        uint64_t* A = spec;
        uint64_t* B = spec + words;
        spec += 2 * words;
        const uint32_t nt = p->logN <= 11 ? 1u : (1u << (p->logN - 11));
        for (uint32_t poly = 0; poly < it.n_polys; ++poly) {
            for (uint32_t l = 0; l < p->n_limbs; ++l) {
                const uint64_t off = ((uint64_t)poly * p->n_limbs + l) << p->logN;
                const LimbDev* lc = p->d_limbs + l;
                const uint8_t lg = (uint8_t)p->logN, single = (uint8_t)(k2 < 0);
                for (uint32_t t = 0; t < nt; ++t) {
                    // forward: a -> A, b -> B (column/single pass first), out range [0, 4q)
                    fA[nfA++] = RagTile{it.d_a + off, A + off, lc, t, (uint8_t)k1, lg, single, 4};
                    fA[nfA++] = RagTile{it.d_b + off, B + off, lc, t, (uint8_t)k1, lg, single, 4};
                    if (!single) {
                        fB[nfB++] = RagTile{A + off, A + off, lc, t, (uint8_t)k2, lg, 1, 4};
                        fB[nfB++] = RagTile{B + off, B + off, lc, t, (uint8_t)k2, lg, 1, 4};
                    }
                    // inverse of A B (the product in the first pass's staging):
                    // -> result (row/single pass first), out range [0, q)
                    iA[niA++] = MulRagTile{A + off, B + off, it.d_result + off, lc, t,
                                           (uint8_t)(single ? k1 : k2), lg, single, 1, 0};
                    if (!single)
                        iB[niB++] = RagTile{it.d_result + off, it.d_result + off, lc, t,
                                            (uint8_t)k1, lg, 1, 1};
                }
            }
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool staged =
        cudaMemsetAsync(counters, 0, 4 * sizeof(uint32_t), s) == cudaSuccess &&
        cudaMemcpyAsync(ws + L.tiles_off, stage->buf, host_bytes, cudaMemcpyHostToDevice, s) ==
            cudaSuccess &&
        cudaEventRecord(stage->done, s) == cudaSuccess;
    if (!staged) return HX_ERR_CUDA;   // stays busy: an enqueued copy may still read it
    staging_release(stage);
    const RagTile* dt = (const RagTile*)(ws + L.tiles_off);
    const int gf = rag_grid(true), gi = rag_grid(false);
    auto pass = [&](bool fwd, const RagTile* t, uint64_t cnt, uint32_t* ctr, int grid) {
        if (!cnt) return cudaSuccess;
        const unsigned g = (unsigned)std::min<uint64_t>(cnt, (uint64_t)grid);
        if (fwd)
            ragged_pass_kernel<true><<<g, 256, kRagSmem, s>>>(t, (uint32_t)cnt, ctr);
        else
            ragged_pass_kernel<false><<<g, 256, kRagSmem, s>>>(t, (uint32_t)cnt, ctr);
        count_launch();
        return cudaGetLastError();
    };
    cudaError_t e = pass(true, dt, L.fA, counters, gf);
    if (e == cudaSuccess) e = pass(true, dt + L.fA, L.fB, counters + 1, gf);
    if (e == cudaSuccess && L.iA) {
        const MulRagTile* dm = (const MulRagTile*)(dt + L.fA + L.fB + L.iB);
        const unsigned g = (unsigned)std::min<uint64_t>(L.iA, (uint64_t)rag_mul_grid());
        ragged_mul_inv_kernel<<<g, 256, kRagSmem, s>>>(dm, (uint32_t)L.iA, counters + 2);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = pass(false, dt + L.fA + L.fB, L.iB, counters + 3, gi);
    return e == cudaSuccess ? HX_OK : HX_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Ragged transforms in a caller-provided workspace (the serving primitive for
// NTT requests): the set of hx_batch_create, run once like
// hx_batch_run_static, with the counters and the tile list in the caller's
// workspace instead of the library's fixed array, so calls on different
// streams, each with its own workspace, may overlap.
// ---------------------------------------------------------------------------
static const uint64_t kNttWsHeader = 256;   // the two work counters

extern "C" int hx_ntt_ragged_workspace(const hx_ragged_item* items, uint32_t n_items,
                                       uint64_t* bytes) {
    if (!bytes) return HX_ERR_NULL;
    uint64_t n_first = 0, n_second = 0;
    int st = rag_check_count(items, n_items, 1, 1, 1, &n_first, &n_second);
    if (st != HX_OK) return st;
    if (n_first > 0xffffffffull || n_second > 0xffffffffull) return HX_ERR_CAPACITY;
    const uint64_t b = kNttWsHeader + (n_first + n_second) * sizeof(RagTile);
    *bytes = (b + 255) & ~255ull;
    return HX_OK;
}

extern "C" int hx_ntt_ragged(const hx_ragged_item* items, uint32_t n_items, uint32_t direction,
                             uint32_t in_mf, uint32_t out_mf, void* d_workspace,
                             uint64_t workspace_bytes, hx_stream_t stream) {
    if (!d_workspace) return HX_ERR_NULL;
    if ((uintptr_t)d_workspace & 255u) return HX_ERR_ALIGN;
    uint64_t n_first = 0, n_second = 0;
    int st = rag_check_count(items, n_items, direction, in_mf, out_mf, &n_first, &n_second);
    if (st != HX_OK) return st;
    if (n_first > 0xffffffffull || n_second > 0xffffffffull) return HX_ERR_CAPACITY;
    const uint64_t tile_bytes = (n_first + n_second) * sizeof(RagTile);
    if (workspace_bytes < kNttWsHeader + tile_bytes) return HX_ERR_CAPACITY;
    int dev = 0;
    cudaGetDevice(&dev);
    DescStaging* stage = staging_acquire(tile_bytes, dev);
    if (!stage) return HX_ERR_NOMEM;
    const bool fwd = direction == 1;
    rag_fill(items, n_items, fwd, out_mf, (RagTile*)stage->buf);
    unsigned char* ws = (unsigned char*)d_workspace;
    uint32_t* counters = (uint32_t*)ws;
    RagTile* d_tiles = (RagTile*)(ws + kNttWsHeader);
    cudaStream_t s = (cudaStream_t)stream;
    const bool staged =
        cudaMemsetAsync(counters, 0, 2 * sizeof(uint32_t), s) == cudaSuccess &&
        cudaMemcpyAsync(d_tiles, stage->buf, tile_bytes, cudaMemcpyHostToDevice, s) ==
            cudaSuccess &&
        cudaEventRecord(stage->done, s) == cudaSuccess;
    if (!staged) return HX_ERR_CUDA;   // stays busy: an enqueued copy may still read it
    staging_release(stage);
    return rag_launch(fwd, d_tiles, n_first, n_second, counters, s);
}
