// Host side of the NTT: schedule validation and pass launches.  The kernels
// are in ntt_kernels.cuh (instantiated in ntt_fwd.cu and ntt_inv.cu).
//
// A schedule (NttCfg) splits the log2 N stages into one or two passes; each
// pass is one kernel launch.  Plain passes launch one block per (tile,
// polynomial, limb); pipelined passes launch a persistent grid of as many
// blocks as fit on the GPU at once, each walking tiles with double
// buffering.  The forward transform runs the passes in stage order, the
// inverse in reverse.
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "ntt_cluster.cuh"
#include "ntt_kernels.cuh"
#include "ntt_tensor.h"

namespace hx {

// ---------------------------------------------------------------------------
// Cluster-fused schedules (ntt_cluster.cuh): two passes, both with pipe 3,
//   {0, K1, 0, logGc, logR, 3, 1}, {K1, K2, logGb, 0, logR, 3, 1},
// run as ONE launch of clusters of 2^LOG_C CTAs, LOG_C = K2 - logGc =
// K1 - logGb: the first pass's tile is a CTA's column-phase tile, the
// second's its row-phase tile, both N / 2^LOG_C elements.
struct ClusterShape {
    int K1, K2, logR, logC, logGc;
    uint32_t threads;
    size_t smem;
};

static bool is_cluster(const NttCfg& c) {
    return c.npass == 2 && (c.pass[0].pipe == 3 || c.pass[1].pipe == 3);
}

// The kernel's shared-memory allowance is set at every launch: one kernel
// serves several cluster sizes, each with its own tile size.
static cudaError_t cluster_attrs(const void* k, const ClusterShape& s) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)s.smem);
    if (e == cudaSuccess && s.logC > 3)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

// Whether clusters of this shape can be resident at all on the current
// device (shared memory and registers per SM, cluster size); cached.
static bool cluster_fits(const void* k, const ClusterShape& s) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, size_t>, bool> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(k, dev, s.logC, s.smem);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    bool ok = cluster_attrs(k, s) == cudaSuccess;
    if (ok) {
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1u << s.logC;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.gridDim = dim3(1u << s.logC, 1, 1);
        lc.blockDim = dim3(s.threads, 1, 1);
        lc.dynamicSmemBytes = s.smem;
        lc.attrs = at;
        lc.numAttrs = 1;
        int n = 0;
        ok = cudaOccupancyMaxActiveClusters(&n, k, &lc) == cudaSuccess && n > 0;
    }
    cudaGetLastError();   // a refused query leaves no error behind
    cache[key] = ok;
    return ok;
}

// Shape of a cluster-fused schedule; false if `c` is not one the library can
// run (kind: 0 forward, 1 inverse, 2 tensor-fused inverse).
static bool cluster_shape(int L, const NttCfg& c, int kind, ClusterShape* out) {
    if (c.npass != 2) return false;
    const PassCfg& a = c.pass[0];
    const PassCfg& b = c.pass[1];
    if (a.pipe != 3 || b.pipe != 3 || a.np != 1 || b.np != 1 || a.logR != b.logR) return false;
    if (a.s0 != 0 || a.logGb != 0 || b.s0 != a.K || b.logGc != 0 || a.K + b.K != L) return false;
    ClusterShape s;
    s.K1 = a.K;
    s.K2 = b.K;
    s.logR = a.logR;
    s.logGc = a.logGc;
    s.logC = b.K - a.logGc;
    if (s.logC != a.K - b.logGb || s.logC < 1 || s.logC > 4) return false;
    if (a.logGc < 2 || b.logGb < 0) return false;   // >= 32-byte column segments in HBM
    const int logE = L - s.logC, logT = logE - s.logR;
    if (logT < 5 || logT > 10) return false;         // 32 .. 1024 threads
    s.threads = 1u << logT;
    s.smem = (size_t)8 * padded(1u << logE);
    if (s.smem > 200 * 1024) return false;
    const void* k = kind == 0   ? (const void*)pick_cluster_f(s.logR, s.K1, s.K2)
                    : kind == 1 ? (const void*)pick_cluster_i(s.logR, s.K1, s.K2)
                                : (const void*)pick_cluster_t(s.logR, s.K1, s.K2);
    if (!k || !cluster_fits(k, s)) return false;
    if (out) *out = s;
    return true;
}

static cudaLaunchConfig_t cluster_launch_cfg(const ClusterShape& s, dim3 grid, cudaStream_t st,
                                             cudaLaunchAttribute* at) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1u << s.logC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = dim3(s.threads, 1, 1);
    lc.dynamicSmemBytes = s.smem;
    lc.stream = st;
    lc.attrs = at;
    lc.numAttrs = 1;
    return lc;
}

// Kernel id of a cluster launch for launch timing: kind 3, bit 2 forward,
// bits 4-6 logR, 7-11 K1, bit 12 tensor-fused, 15-19 K2.
static uint32_t cluster_kernel_id(bool fwd, bool tensor, const ClusterShape& s) {
    return 3u | (fwd ? 4u : 0u) | ((uint32_t)s.logR << 4) | ((uint32_t)s.K1 << 7) |
           (tensor ? 1u << 12 : 0u) | ((uint32_t)s.K2 << 15);
}

static cudaError_t launch_cluster(const hx_plan_s* plan, const NttCfg& cfg, uint64_t* out,
                                  const uint64_t* in, uint32_t n_polys, bool forward,
                                  uint32_t out_mf, cudaStream_t stream) {
    ClusterShape s;
    if (!cluster_shape(plan->logN, cfg, forward ? 0 : 1, &s)) return cudaErrorInvalidConfiguration;
    PassArgs a{};
    a.out = out;
    a.in = in;
    a.limbs = plan->d_limbs;
    a.order = plan->d_order;   // few long blocks: the costliest limbs start first
    a.n_limbs = plan->n_limbs;
    a.n_polys = n_polys;
    a.L = plan->logN;
    a.s0 = 0;
    a.logGb = s.K1 - s.logC;
    a.logGc = s.logGc;
    a.log_tiles_c = 0;
    a.last = 1;
    a.out_mf = out_mf;
    ClusterKernel k = forward ? pick_cluster_f(s.logR, s.K1, s.K2)
                              : pick_cluster_i(s.logR, s.K1, s.K2);
    cudaError_t e = cluster_attrs((const void*)k, s);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t lc =
        cluster_launch_cfg(s, dim3(n_polys << s.logC, plan->n_limbs, 1), stream, at);
    const uint32_t slot = timing_begin(stream, cluster_kernel_id(forward, false, s));
    e = cudaLaunchKernelEx(&lc, k, a);
    timing_end(slot, stream);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

static PassKernel pick(bool fwd, const PassCfg& p) {
    const bool column = p.logGc > 0;
    if (p.pipe == 1)
        return p.np != 1 ? nullptr
                         : fwd ? pick_pipe_f(column, p.logR, p.K) : pick_pipe_i(column, p.logR, p.K);
    if (p.pipe == 2) {
        if (p.np == 2)
            return fwd ? pick_tws_f2(column, p.logR, p.K) : pick_tws_i2(column, p.logR, p.K);
        if (p.np == 1)
            return fwd ? pick_tws_f1(column, p.logR, p.K) : pick_tws_i1(column, p.logR, p.K);
        return nullptr;
    }
    if (p.np == 2)
        return fwd ? pick_plain_f2(column, p.logR, p.K) : pick_plain_i2(column, p.logR, p.K);
    if (p.np == 1)
        return fwd ? pick_plain_f1(column, p.logR, p.K) : pick_plain_i1(column, p.logR, p.K);
    return nullptr;
}

// Dynamic shared memory of one block of a pass: the persistent kernel's two
// tile buffers; the per-tile kernels' NP padded data tiles, plus the staged
// twiddle pairs in mode 2.
static size_t pass_smem(const PassCfg& p) {
    const int logTE = p.logGb + p.K + p.logGc;
    if (p.pipe == 1) return (size_t)16 << logTE;
    size_t b = (size_t)8 * p.np * padded(1u << logTE);
    if (p.pipe == 2) b += 16 * (size_t)staged_twiddles(p.logGb, p.K);
    return b;
}

static bool pass_ok(int L, const PassCfg& p) {
    if (p.pipe < 0 || p.pipe > 2) return false;
    if (!pick(true, p) || !pick(false, p)) return false;
    const int w = L - p.s0 - p.K;
    if (w < 0 || p.s0 < 0) return false;
    if (w == 0 && p.logGc != 0) return false;
    if (w > 0 && (p.logGc < 2 || p.logGc > w)) return false;   // >= 32-byte row segments
    if (p.logGb < 0 || p.logGb > p.s0) return false;
    if (w > 0 && p.logGb != 0) return false;
    const int logTE = p.logGb + p.K + p.logGc;
    const int logT = logTE - p.logR;
    if (logT < 5 || logT > (p.pipe == 1 ? 8 : 9)) return false;   // 32 .. 256 / 512 threads
    if (pass_smem(p) > 192 * 1024) return false;
    return true;
}

bool cfg_supported(int L, const NttCfg& cfg) {
    if (is_cluster(cfg))
        return cluster_shape(L, cfg, 0, nullptr) && cluster_shape(L, cfg, 1, nullptr);
    if (cfg.npass < 1 || cfg.npass > 2) return false;
    int s = 0;
    for (int i = 0; i < cfg.npass; ++i) {
        if (cfg.pass[i].s0 != s || !pass_ok(L, cfg.pass[i])) return false;
        s += cfg.pass[i].K;
    }
    return s == L;
}

// Resident blocks per SM of a pipelined kernel, cached per (kernel, device).
static int resident_blocks(PassKernel k, int threads, size_t smem, int* sms) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, std::pair<int, int>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair((const void*)k, dev);
    auto it = cache.find(key);
    if (it == cache.end()) {
        int per_sm = 0, n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        it = cache.emplace(key, std::make_pair(per_sm > 0 ? per_sm : 1, n > 0 ? n : 1)).first;
    }
    *sms = it->second.second;
    return it->second.first;
}

// Kernel id of a pass for launch timing (layout in hx_internal.h).
static uint32_t pass_kernel_id(bool fwd, const PassCfg& p, bool mul = false) {
    return (p.pipe == 1 ? 1u : 0u) | (fwd ? 4u : 0u) | (p.logGc > 0 ? 8u : 0u) |
           ((uint32_t)p.logR << 4) | ((uint32_t)p.K << 7) | ((uint32_t)p.np << 12) |
           (p.pipe == 2 ? 1u << 14 : 0u) | (mul ? 1u << 15 : 0u);
}

// Launches one pass of a schedule over n_polys polynomials.  With mul_b the
// pass is the inverse's first (row) pass with the dyadic product of `in`
// and mul_b (both below mul_mf q) computed in its staging step.
static cudaError_t launch_pass(const hx_plan_s* plan, const PassCfg& p, uint64_t* out,
                               const uint64_t* in, uint32_t n_polys, bool forward, bool last,
                               uint32_t out_mf, cudaStream_t stream,
                               const uint64_t* mul_b = nullptr, uint32_t mul_mf = 1) {
    const int L = plan->logN;
    PassArgs a;
    a.out = out;
    a.in = in;
    a.limbs = plan->d_limbs;
    // column passes: fewer, longer blocks (16 elements a thread) -- the costliest
    // limbs start first; row passes: many short blocks, natural order
    a.order = p.logGc > 0 ? plan->d_order : nullptr;
    a.n_limbs = plan->n_limbs;
    a.n_polys = n_polys;
    a.L = L;
    a.s0 = p.s0;
    a.logGb = p.logGb;
    a.logGc = p.logGc;
    a.log_tiles_c = (L - p.s0 - p.K) - p.logGc;
    a.last = last;
    a.out_mf = out_mf;
    const int logTE = p.logGb + p.K + p.logGc;
    const uint32_t tiles = 1u << (L - logTE);
    const uint32_t threads = 1u << (logTE - p.logR);
    const size_t smem = pass_smem(p);
    PassKernel k = pick(forward, p);
    if (!k) return cudaErrorInvalidConfiguration;
    MulPassKernel km = nullptr;
    if (mul_b) {
        if (forward || p.pipe == 1 || p.logGc != 0) return cudaErrorInvalidConfiguration;
        km = pick_mul_inv(p.logR, p.K, p.np, p.pipe == 2);
        if (!km) return cudaErrorInvalidConfiguration;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(km ? (const void*)km : (const void*)k,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (km) {
        dim3 grid(tiles * ((n_polys + p.np - 1) / p.np), plan->n_limbs);
        const uint32_t slot = timing_begin(stream, pass_kernel_id(false, p, true));
        km<<<grid, threads, smem, stream>>>(a, mul_b, mul_mf);
        timing_end(slot, stream);
    } else if (p.pipe == 1) {
        int sms = 0;
        const int per_sm = resident_blocks(k, threads, smem, &sms);
        const uint64_t total = (uint64_t)tiles * n_polys * plan->n_limbs;
        const uint64_t grid = std::min<uint64_t>(total, (uint64_t)per_sm * sms);
        const uint32_t slot = timing_begin(stream, pass_kernel_id(forward, p));
        k<<<(unsigned)grid, threads, smem, stream>>>(a);
        timing_end(slot, stream);
    } else {
        dim3 grid(tiles * ((n_polys + p.np - 1) / p.np), plan->n_limbs);
        const uint32_t slot = timing_begin(stream, pass_kernel_id(forward, p));
        k<<<grid, threads, smem, stream>>>(a);
        timing_end(slot, stream);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ntt(const hx_plan_s* plan, uint64_t* out, const uint64_t* in,
                       uint32_t n_polys, bool forward, uint32_t in_mf, uint32_t out_mf,
                       const NttCfg& cfg, cudaStream_t stream) {
    (void)in_mf;  // every allowed input range is inside the butterflies' lazy range
    if (is_cluster(cfg))
        return launch_cluster(plan, cfg, out, in, n_polys, forward, out_mf, stream);
    for (int step = 0; step < cfg.npass; ++step) {
        const int pi = forward ? step : cfg.npass - 1 - step;
        cudaError_t e = launch_pass(plan, cfg.pass[pi], out, step == 0 ? in : out, n_polys,
                                    forward, step == cfg.npass - 1, out_mf, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool mul_fusable(const NttCfg& cfg) {
    if (is_cluster(cfg)) return false;
    const PassCfg& p = cfg.pass[cfg.npass - 1];   // the inverse runs this pass first
    return p.pipe != 1 && p.logGc == 0 && pick_mul_inv(p.logR, p.K, p.np, p.pipe == 2);
}

cudaError_t launch_mul_inverse(const hx_plan_s* plan, uint64_t* out, const uint64_t* a,
                               const uint64_t* b, uint32_t n_polys, uint32_t in_mf,
                               const NttCfg& cfg, cudaStream_t stream) {
    if (!mul_fusable(cfg)) return cudaErrorNotSupported;
    const int first = cfg.npass - 1;
    cudaError_t e = launch_pass(plan, cfg.pass[first], out, a, n_polys, false, cfg.npass == 1, 1,
                                stream, b, in_mf);
    if (e != cudaSuccess || cfg.npass == 1) return e;
    return launch_pass(plan, cfg.pass[0], out, out, n_polys, false, true, 1, stream);
}

// The fused pass takes the first inverse pass's shape; a schedule with two
// polynomials per thread there selects the kernel that computes and
// transforms all three outputs of a ciphertext in one block.
static int tensor_npf(const PassCfg& p) { return p.np > 1 ? 3 : 1; }

// The plan's launch order permutes limbs within runs of 64, so every chunk of
// the fused pass's launches maps onto itself.
static_assert(kTensorLimbs == 64, "launch_order permutes within runs of kTensorLimbs");

// One cluster-fused launch per 64 limbs: the tensor's element-wise step in
// the inverse's first (row) phase, then the whole inverse transform.
static cudaError_t launch_cluster_tensor(const hx_plan_s* plan, uint64_t* out, const uint64_t* A,
                                         const uint64_t* E, uint32_t n_ct,
                                         const uint64_t* h_scalars, uint32_t in_mf,
                                         const NttCfg& cfg, cudaStream_t stream) {
    ClusterShape s;
    if (!cluster_shape(plan->logN, cfg, 2, &s)) return cudaErrorInvalidConfiguration;
    PassArgs a{};
    a.out = out;
    a.in = nullptr;
    a.limbs = plan->d_limbs;
    a.order = plan->d_order;
    a.n_limbs = plan->n_limbs;
    a.n_polys = 3 * n_ct;
    a.L = plan->logN;
    a.logGb = s.K1 - s.logC;
    a.logGc = s.logGc;
    a.last = 1;
    a.out_mf = 1;
    ClusterTensorKernel k = pick_cluster_t(s.logR, s.K1, s.K2);
    const cudaError_t ea = cluster_attrs((const void*)k, s);
    if (ea != cudaSuccess) return ea;
    for (uint32_t limb0 = 0; limb0 < plan->n_limbs; limb0 += kTensorLimbs) {
        const uint32_t chunk = std::min<uint32_t>(kTensorLimbs, plan->n_limbs - limb0);
        TensorIn t{};
        t.A = A;
        t.E = E;
        t.n_ct = n_ct;
        t.in_mf = in_mf;
        t.limb0 = limb0;
        for (uint32_t i = 0; i < chunk; ++i) {
            const uint64_t q = plan->moduli[limb0 + i], sc = h_scalars[limb0 + i];
            t.s[i] = sc;
            t.sp[i] = (uint64_t)(((unsigned __int128)sc << 64) / q);
        }
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t lc =
            cluster_launch_cfg(s, dim3((3 * n_ct) << s.logC, chunk, 1), stream, at);
        const uint32_t slot = timing_begin(stream, cluster_kernel_id(false, true, s));
        cudaError_t e = cudaLaunchKernelEx(&lc, k, a, t);
        timing_end(slot, stream);
        count_launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool tensor_fusable(const NttCfg& cfg) {
    if (is_cluster(cfg)) {
        const int L = cfg.pass[0].K + cfg.pass[1].K;
        return cluster_shape(L, cfg, 2, nullptr);
    }
    const PassCfg& p = cfg.pass[cfg.npass - 1];   // the inverse runs this pass first
    if (p.pipe == 1 || p.logGc != 0) return false;
    if (!pick_tensor_inv(p.logR, p.K, p.pipe == 2, tensor_npf(p))) return false;
    const int logTE = p.logGb + p.K;
    const size_t smem = (size_t)8 * tensor_npf(p) * padded(1u << logTE) +
                        (p.pipe == 2 ? 16 * (size_t)staged_twiddles(p.logGb, p.K) : 0);
    return smem <= 192 * 1024;
}

cudaError_t launch_tensor_inverse(const hx_plan_s* plan, uint64_t* out, const uint64_t* A,
                                  const uint64_t* E, uint32_t n_ct, const uint64_t* h_scalars,
                                  uint32_t in_mf, const NttCfg& cfg, cudaStream_t stream) {
    if (!tensor_fusable(cfg)) return cudaErrorNotSupported;
    if (is_cluster(cfg))
        return launch_cluster_tensor(plan, out, A, E, n_ct, h_scalars, in_mf, cfg, stream);
    const int L = plan->logN;
    const PassCfg& p = cfg.pass[cfg.npass - 1];
    const int npf = tensor_npf(p);
    TensorPassKernel k = pick_tensor_inv(p.logR, p.K, p.pipe == 2, npf);
    PassArgs a;
    a.out = out;
    a.in = nullptr;
    a.limbs = plan->d_limbs;
    a.order = plan->d_order;   // few long blocks: the costliest limbs start first
    a.n_limbs = plan->n_limbs;
    a.n_polys = 3 * n_ct;
    a.L = L;
    a.s0 = p.s0;
    a.logGb = p.logGb;
    a.logGc = 0;
    a.log_tiles_c = 0;
    a.last = cfg.npass == 1;
    a.out_mf = 1;
    const int logTE = p.logGb + p.K;
    const uint32_t tiles = 1u << (L - logTE);
    const uint32_t threads = 1u << (logTE - p.logR);
    const size_t smem = (size_t)8 * npf * padded(1u << logTE) +
                        (p.pipe == 2 ? 16 * (size_t)staged_twiddles(p.logGb, p.K) : 0);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    for (uint32_t limb0 = 0; limb0 < plan->n_limbs; limb0 += kTensorLimbs) {
        const uint32_t chunk = std::min<uint32_t>(kTensorLimbs, plan->n_limbs - limb0);
        TensorIn t{};
        t.A = A;
        t.E = E;
        t.n_ct = n_ct;
        t.in_mf = in_mf;
        t.limb0 = limb0;
        for (uint32_t i = 0; i < chunk; ++i) {
            const uint64_t q = plan->moduli[limb0 + i], sc = h_scalars[limb0 + i];
            t.s[i] = sc;
            t.sp[i] = (uint64_t)(((unsigned __int128)sc << 64) / q);
        }
        const uint32_t slot = timing_begin(
            stream, 2u | ((uint32_t)p.logR << 4) | ((uint32_t)p.K << 7) | ((uint32_t)npf << 12) |
                        (p.pipe == 2 ? 1u << 14 : 0u));
        k<<<dim3(tiles * (npf == 3 ? 1 : 3) * n_ct, chunk), threads, smem, stream>>>(a, t);
        timing_end(slot, stream);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (cfg.npass == 2)
        return launch_pass(plan, cfg.pass[0], out, out, 3 * n_ct, false, true, 1, stream);
    return cudaSuccess;
}


// The step's two row passes fused around the tensor (ntt_ctrow.cu): both
// schedules two-pass, their row passes over the same stages with 8 elements
// a thread; the kernel runs both in the inverse's row tiles.
bool ct_step_fusable(const NttCfg& f, const NttCfg& i) {
    if (f.npass != 2 || i.npass != 2 || is_cluster(f) || is_cluster(i)) return false;
    const PassCfg& fr = f.pass[1];
    const PassCfg& ir = i.pass[1];
    if (fr.logGc != 0 || ir.logGc != 0 || fr.s0 != ir.s0 || fr.K != ir.K || fr.logR != 3 ||
        ir.logR != 3)
        return false;
    if (!pick_ct_row(3, ir.K)) return false;
    const int logT = ir.logGb + ir.K - 3;
    return logT >= 5 && logT <= 9 &&
           (size_t)8 * 4 * padded(1u << (ir.logGb + ir.K)) <= 192 * 1024;
}

cudaError_t launch_ct_step(const hx_plan_s* plan, uint64_t* out, const uint64_t* in,
                           uint64_t* work, const uint64_t* E, uint32_t n_ct,
                           const uint64_t* h_scalars, const NttCfg& f, const NttCfg& i,
                           cudaStream_t stream) {
    if (!ct_step_fusable(f, i)) return cudaErrorNotSupported;
    const int L = plan->logN;
    // the forward's column pass over the four operands
    cudaError_t e = launch_pass(plan, f.pass[0], work, in, 4 * n_ct, true, false, 4, stream);
    if (e != cudaSuccess) return e;
    const PassCfg& p = i.pass[1];   // the row tile of both directions
    TensorPassKernel k = pick_ct_row(3, p.K);
    PassArgs a{};
    a.out = out;
    a.in = nullptr;
    a.limbs = plan->d_limbs;
    a.order = plan->d_order;   // few long blocks: the costliest limbs start first
    a.n_limbs = plan->n_limbs;
    a.n_polys = 3 * n_ct;
    a.L = L;
    a.s0 = p.s0;
    a.logGb = p.logGb;
    a.logGc = 0;
    a.log_tiles_c = 0;
    a.last = 0;
    a.out_mf = 1;
    const int logTE = p.logGb + p.K;
    const uint32_t tiles = 1u << (L - logTE);
    const uint32_t threads = 1u << (logTE - 3);
    const size_t smem = (size_t)8 * 4 * padded(1u << logTE);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
    }
    for (uint32_t limb0 = 0; limb0 < plan->n_limbs; limb0 += kTensorLimbs) {
        const uint32_t chunk = std::min<uint32_t>(kTensorLimbs, plan->n_limbs - limb0);
        TensorIn t{};
        t.A = work;
        t.E = E;
        t.n_ct = n_ct;
        t.in_mf = 4;
        t.limb0 = limb0;
        for (uint32_t l = 0; l < chunk; ++l) {
            const uint64_t q = plan->moduli[limb0 + l], sc = h_scalars[limb0 + l];
            t.s[l] = sc;
            t.sp[l] = (uint64_t)(((unsigned __int128)sc << 64) / q);
        }
        const uint32_t slot =
            timing_begin(stream, 2u | (3u << 4) | ((uint32_t)p.K << 7) | (1u << 16));
        k<<<dim3(tiles * n_ct, chunk), threads, smem, stream>>>(a, t);
        timing_end(slot, stream);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // the inverse's column pass over the three outputs, N^-1 folded
    return launch_pass(plan, i.pass[0], out, out, 3 * n_ct, false, true, 1, stream);
}

// The product's step kernel runs the forward's and the inverse's row stages
// in the inverse's row tiles: both schedules two-pass with the same split,
// 8 elements a thread in both row passes.
bool mul_step_fusable(const NttCfg& f, const NttCfg& i) {
    if (f.npass != 2 || i.npass != 2 || is_cluster(f) || is_cluster(i)) return false;
    const PassCfg& fr = f.pass[1];
    const PassCfg& ir = i.pass[1];
    if (fr.logGc != 0 || ir.logGc != 0 || fr.s0 != ir.s0 || fr.K != ir.K || fr.logR != 3 ||
        ir.logR != 3)
        return false;
    if (!pick_mul_row(3, ir.K)) return false;
    const int logT = ir.logGb + ir.K - 3;
    return logT >= 5 && logT <= 9 &&
           (size_t)8 * 2 * padded(1u << (ir.logGb + ir.K)) <= 192 * 1024;
}

cudaError_t launch_mul_step(const hx_plan_s* plan, uint64_t* out, const uint64_t* a,
                            const uint64_t* b, uint64_t* work, uint32_t n_polys,
                            const NttCfg& f, const NttCfg& i, cudaStream_t stream) {
    if (!mul_step_fusable(f, i)) return cudaErrorNotSupported;
    const int L = plan->logN;
    const uint64_t S = (uint64_t)n_polys * plan->n_limbs << L;
    // the forward's column pass over a, then b, into the two halves of work
    cudaError_t e = launch_pass(plan, f.pass[0], work, a, n_polys, true, false, 4, stream);
    if (e != cudaSuccess) return e;
    e = launch_pass(plan, f.pass[0], work + S, b, n_polys, true, false, 4, stream);
    if (e != cudaSuccess) return e;
    const PassCfg& p = i.pass[1];
    PassKernel k = pick_mul_row(3, p.K);
    PassArgs args{};
    args.out = out;
    args.in = work;
    args.limbs = plan->d_limbs;
    args.order = plan->d_order;
    args.n_limbs = plan->n_limbs;
    args.n_polys = n_polys;
    args.L = L;
    args.s0 = p.s0;
    args.logGb = p.logGb;
    args.logGc = 0;
    args.log_tiles_c = 0;
    args.last = 0;
    args.out_mf = 1;
    const int logTE = p.logGb + p.K;
    const uint32_t tiles = 1u << (L - logTE);
    const size_t smem = (size_t)8 * 2 * padded(1u << logTE);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint32_t slot =
        timing_begin(stream, 2u | (3u << 4) | ((uint32_t)p.K << 7) | (3u << 16));
    k<<<dim3(tiles * n_polys, plan->n_limbs), 1u << (logTE - 3), smem, stream>>>(args);
    timing_end(slot, stream);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the inverse's column pass, N^-1 folded
    return launch_pass(plan, i.pass[0], out, out, n_polys, false, true, 1, stream);
}
}  // namespace hx
