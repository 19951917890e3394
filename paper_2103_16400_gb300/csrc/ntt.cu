// Fused negacyclic NTT passes for sm_103a.
//
// The forward transform is the radix-2 Cooley-Tukey NTT of Section 2.2 with
// the Harvey butterfly (values kept lazily in [0, 4q)); the inverse is the
// radix-2 Gentleman-Sande InvNTT with the Harvey inverse butterfly (values in
// [0, 2q)) and the N^-1 scaling folded into its last stage.  Both index the
// twiddles exactly as the paper's algorithms do: stage s (s = 0 .. log2 N - 1,
// m = 2^s) pairs element j with j + N/2^(s+1), and uses table entry
// 2^s + (j >> (log2 N - s)) -- psi_rev for the forward, psi^-1_rev for the
// inverse, where the Gentleman-Sande loop runs the same stages in reverse.
//
// GPU design (not the paper's AVX512 one): a pass takes K consecutive stages
// for a tile of 2^logGb x 2^K x 2^logGc elements that those stages keep
// closed (fixed top index bits b, fixed low index bits c).  The tile moves
// HBM -> shared memory once, coalesced in 16-byte vectors, then runs in
// register rounds of up to 2^LOG_R elements per thread (LOG_R stages per
// round, butterflies entirely in registers), exchanging through an XOR-
// swizzled shared-memory tile between rounds, and goes back to HBM once.
// N <= 2^13 is one pass (one HBM read and write per coefficient); larger N
// takes two passes (a column pass over the first stages, a row pass over
// contiguous chunks for the rest).  Limbs with q < 2^30 compute on 32-bit
// words (three 32-bit multiplies per butterfly instead of fifteen).
#include <stdint.h>

#include "hx_internal.h"
#include "modarith.cuh"

namespace hx {

struct PassArgs {
    uint64_t* out;
    const uint64_t* in;
    const LimbDev* limbs;
    uint32_t n_limbs;
    uint32_t n_polys;
    int L;          // log2 N
    int s0;         // first stage of the pass
    int logGb;      // log2 of top-index values per tile
    int logGc;      // log2 of low-index values per tile (0 when the pass ends at stage L-1)
    int log_tiles_c;
    uint32_t last;   // this pass finishes the transform
    uint32_t out_mf; // output mod factor (applied when last)
};

// Round schedule of a pass: K stages split into ceil(K / LOG_R) rounds of
// near-equal size; round i covers e-bits [off(i), off(i) + size(i)) counted
// from the top (the first stage of the pass acts on the top e-bit).
template <int K, int LOG_R>
struct Sched {
    static constexpr int NR = (K + LOG_R - 1) / LOG_R;
    __host__ __device__ static constexpr int size(int i) { return K / NR + (i < K % NR ? 1 : 0); }
    __host__ __device__ static constexpr int off(int i) {
        int s = 0;
        for (int j = 0; j < i; ++j) s += size(j);
        return s;
    }
};

// Shared-memory tile position of local element l: XOR the 16-word bank group
// with bits 4..7 so that both column-wise and stride-2^r row-wise accesses
// of a half-warp land in distinct 8-byte banks.
__device__ __forceinline__ uint32_t swz(uint32_t l) { return l ^ ((l >> 4) & 15u); }

template <typename Wd>
struct Word;

template <>
struct Word<uint64_t> {
    static __device__ __forceinline__ void fwd(uint64_t& a, uint64_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t q2) {
        harvey_fwd64(a, b, w.x, w.y, q, q2);
    }
    static __device__ __forceinline__ void inv(uint64_t& a, uint64_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t q2) {
        harvey_inv64(a, b, w.x, w.y, q, q2);
    }
    static __device__ __forceinline__ uint64_t mul(uint64_t x, uint64_t w, uint64_t wp,
                                                   uint64_t q) {
        return shoup_mul_lazy64(x, w, wp, q);
    }
};

template <>
struct Word<uint32_t> {
    static __device__ __forceinline__ void fwd(uint32_t& a, uint32_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t q2) {
        harvey_fwd32(a, b, (uint32_t)w.x, (uint32_t)w.y, (uint32_t)q, (uint32_t)q2);
    }
    static __device__ __forceinline__ void inv(uint32_t& a, uint32_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t q2) {
        harvey_inv32(a, b, (uint32_t)w.x, (uint32_t)w.y, (uint32_t)q, (uint32_t)q2);
    }
    static __device__ __forceinline__ uint32_t mul(uint32_t x, uint64_t w, uint64_t wp,
                                                   uint64_t q) {
        return shoup_mul_lazy32(x, (uint32_t)w, (uint32_t)wp, (uint32_t)q);
    }
};

struct RoundCtx {
    uint64_t b_base;   // first top-index value of the tile
    int s0;
    int logGc;
    uint32_t nthreads;
    bool last;
    uint32_t out_mf;
};

// One register round: stages s0+P .. s0+P+R-1 of the pass.  Each thread holds
// 2^LOG_R elements = U = 2^(LOG_R-R) independent groups of 2^R; register
// index reg = (v << (LOG_R - R)) | u, so the pair of sub-stage k differs in
// register bit LOG_R-1-k (a compile-time position).
template <bool FWD, typename Wd, int LOG_R, int K, int P, int R>
__device__ __forceinline__ void ntt_round(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                          const LimbDev& lc, const RoundCtx& c) {
    constexpr int RN = 1 << LOG_R;
    constexpr int U = 1 << (LOG_R - R);
    constexpr int ELO = K - P - R;
    Wd x[RN];
    uint64_t pfx[U];
    uint32_t lbase[U];
    const uint32_t cmask = (1u << c.logGc) - 1;
    const int vshift = ELO + c.logGc;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        uint32_t g = u * c.nthreads + threadIdx.x;
        uint32_t cl = g & cmask;
        uint32_t t1 = g >> c.logGc;
        uint32_t elo = t1 & ((1u << ELO) - 1);
        uint32_t t2 = t1 >> ELO;
        uint32_t ehi = t2 & ((1u << P) - 1);
        uint32_t bl = t2 >> P;
        lbase[u] = (bl << (K + c.logGc)) | (ehi << (K - P + c.logGc)) | (elo << c.logGc) | cl;
        pfx[u] = ((c.b_base + bl) << P) | ehi;
    }
#pragma unroll
    for (int reg = 0; reg < RN; ++reg) {
        const int u = reg & (U - 1), v = reg >> (LOG_R - R);
        x[reg] = (Wd)sm[swz(lbase[u] + ((uint32_t)v << vshift))];
    }
    const uint64_t q = lc.q, q2 = lc.two_q;
    if (FWD) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int s = c.s0 + P + k;
            const int hb = LOG_R - 1 - k;
#pragma unroll
            for (int reg0 = 0; reg0 < RN; ++reg0) {
                if (reg0 & (1 << hb)) continue;
                const int reg1 = reg0 | (1 << hb);
                const int u = reg0 & (U - 1), v0 = reg0 >> (LOG_R - R);
                const uint64_t idx = (1ull << s) + (pfx[u] << k) + (uint64_t)(v0 >> (R - k));
                const ulonglong2 w = __ldg(tw + idx);
                Word<Wd>::fwd(x[reg0], x[reg1], w, q, q2);
            }
        }
        if (c.last && c.out_mf == 1) {
#pragma unroll
            for (int reg = 0; reg < RN; ++reg) {
                Wd y = x[reg];
                y = y >= (Wd)q2 ? y - (Wd)q2 : y;
                y = y >= (Wd)q ? y - (Wd)q : y;
                x[reg] = y;
            }
        }
    } else {
#pragma unroll
        for (int k = R - 1; k >= 0; --k) {
            const int s = c.s0 + P + k;
            const int hb = LOG_R - 1 - k;
            if (P == 0 && k == 0 && c.s0 == 0) {
                // stage 0 of the inverse: fold N^-1 into the last butterfly
#pragma unroll
                for (int reg0 = 0; reg0 < RN; ++reg0) {
                    if (reg0 & (1 << hb)) continue;
                    const int reg1 = reg0 | (1 << hb);
                    Wd a = x[reg0], b = x[reg1];
                    Wd sum = a + b;                    // [0, 4q)
                    Wd dif = a - b + (Wd)q2;           // (0, 4q)
                    x[reg0] = Word<Wd>::mul(sum, lc.ninv, lc.ninv_p, q);
                    x[reg1] = Word<Wd>::mul(dif, lc.ninv_w, lc.ninv_w_p, q);
                }
            } else {
#pragma unroll
                for (int reg0 = 0; reg0 < RN; ++reg0) {
                    if (reg0 & (1 << hb)) continue;
                    const int reg1 = reg0 | (1 << hb);
                    const int u = reg0 & (U - 1), v0 = reg0 >> (LOG_R - R);
                    const uint64_t idx = (1ull << s) + (pfx[u] << k) + (uint64_t)(v0 >> (R - k));
                    const ulonglong2 w = __ldg(tw + idx);
                    Word<Wd>::inv(x[reg0], x[reg1], w, q, q2);
                }
            }
        }
        if (c.last && c.out_mf == 1) {
#pragma unroll
            for (int reg = 0; reg < RN; ++reg) {
                Wd y = x[reg];
                x[reg] = y >= (Wd)q ? y - (Wd)q : y;
            }
        }
    }
#pragma unroll
    for (int reg = 0; reg < RN; ++reg) {
        const int u = reg & (U - 1), v = reg >> (LOG_R - R);
        sm[swz(lbase[u] + ((uint32_t)v << vshift))] = (uint64_t)x[reg];
    }
}

template <bool FWD, typename Wd, int LOG_R, int K, int I>
__device__ __forceinline__ void ntt_rounds(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                           const LimbDev& lc, const RoundCtx& c) {
    using S = Sched<K, LOG_R>;
    constexpr int idx = FWD ? I : S::NR - 1 - I;
    RoundCtx cr = c;
    cr.last = c.last && (I == S::NR - 1);
    ntt_round<FWD, Wd, LOG_R, K, S::off(idx), S::size(idx)>(sm, tw, lc, cr);
    __syncthreads();
    if constexpr (I + 1 < S::NR) ntt_rounds<FWD, Wd, LOG_R, K, I + 1>(sm, tw, lc, c);
}

// Global index of local tile element l.
__device__ __forceinline__ uint64_t tile_gidx(uint32_t l, const PassArgs& a, int K,
                                              uint64_t b_base, uint64_t c_base) {
    const int w = a.L - a.s0 - K;
    if (w == 0) return (b_base << K) + l;
    const uint32_t cl = l & ((1u << a.logGc) - 1);
    const uint32_t rho = l >> a.logGc;
    const uint64_t e = rho & ((1u << K) - 1);
    const uint64_t bl = rho >> K;
    return ((b_base + bl) << (a.L - a.s0)) + (e << w) + c_base + cl;
}

template <bool FWD, int LOG_R, int K>
__global__ void __launch_bounds__(512) ntt_pass_kernel(PassArgs a) {
    extern __shared__ uint64_t sm[];
    const uint32_t limb = blockIdx.y;
    const uint32_t poly = blockIdx.x % a.n_polys;
    const uint32_t tile = blockIdx.x / a.n_polys;
    const LimbDev lc = a.limbs[limb];
    const uint64_t N = 1ull << a.L;
    const uint64_t base = ((uint64_t)poly * a.n_limbs + limb) * N;
    const uint32_t tile_c = tile & ((1u << a.log_tiles_c) - 1);
    const uint32_t tile_b = tile >> a.log_tiles_c;
    const uint64_t b_base = (uint64_t)tile_b << a.logGb;
    const uint64_t c_base = (uint64_t)tile_c << a.logGc;
    const uint32_t TE = 1u << (a.logGb + K + a.logGc);
    const uint32_t nthreads = TE >> LOG_R;

    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(a.in + base);
    for (uint32_t i = threadIdx.x; i < TE / 2; i += nthreads) {
        const uint32_t l = 2 * i;
        const ulonglong2 v = src[tile_gidx(l, a, K, b_base, c_base) >> 1];
        sm[swz(l)] = v.x;
        sm[swz(l + 1)] = v.y;
    }
    __syncthreads();

    RoundCtx c{b_base, a.s0, a.logGc, nthreads, a.last != 0, a.out_mf};
    const ulonglong2* tw = FWD ? lc.fwd : lc.inv;
    if (lc.narrow)
        ntt_rounds<FWD, uint32_t, LOG_R, K, 0>(sm, tw, lc, c);
    else
        ntt_rounds<FWD, uint64_t, LOG_R, K, 0>(sm, tw, lc, c);

    ulonglong2* dst = reinterpret_cast<ulonglong2*>(a.out + base);
    for (uint32_t i = threadIdx.x; i < TE / 2; i += nthreads) {
        const uint32_t l = 2 * i;
        dst[tile_gidx(l, a, K, b_base, c_base) >> 1] = make_ulonglong2(sm[swz(l)], sm[swz(l + 1)]);
    }
}

typedef void (*PassKernel)(PassArgs);

template <bool FWD, int LOG_R>
static PassKernel pick_k(int K) {
    switch (K) {
        case 5: return ntt_pass_kernel<FWD, LOG_R, 5>;
        case 6: return ntt_pass_kernel<FWD, LOG_R, 6>;
        case 7: return ntt_pass_kernel<FWD, LOG_R, 7>;
        case 8: return ntt_pass_kernel<FWD, LOG_R, 8>;
        case 9: return ntt_pass_kernel<FWD, LOG_R, 9>;
        case 10: return ntt_pass_kernel<FWD, LOG_R, 10>;
        case 11: return ntt_pass_kernel<FWD, LOG_R, 11>;
        case 12: return ntt_pass_kernel<FWD, LOG_R, 12>;
        case 13: return ntt_pass_kernel<FWD, LOG_R, 13>;
        default: return nullptr;
    }
}

static PassKernel pick(bool fwd, int logR, int K) {
    if (fwd) {
        if (logR == 3) return pick_k<true, 3>(K);
        if (logR == 4) return pick_k<true, 4>(K);
    } else {
        if (logR == 3) return pick_k<false, 3>(K);
        if (logR == 4) return pick_k<false, 4>(K);
    }
    return nullptr;
}

static bool pass_ok(int L, const PassCfg& p) {
    if (!pick(true, p.logR, p.K)) return false;
    const int w = L - p.s0 - p.K;
    if (w < 0 || p.s0 < 0) return false;
    if (w == 0 && p.logGc != 0) return false;
    if (w > 0 && (p.logGc < 1 || p.logGc > w)) return false;
    if (p.logGb < 0 || p.logGb > p.s0) return false;
    const int logTE = p.logGb + p.K + p.logGc;
    const int logT = logTE - p.logR;
    if (logT < 5 || logT > 9) return false;          // 32 .. 512 threads
    if ((8u << logTE) > 200 * 1024) return false;    // shared-memory tile
    return true;
}

bool cfg_supported(int L, const NttCfg& cfg) {
    if (cfg.npass < 1 || cfg.npass > 2) return false;
    int s = 0;
    for (int i = 0; i < cfg.npass; ++i) {
        if (cfg.pass[i].s0 != s || !pass_ok(L, cfg.pass[i])) return false;
        s += cfg.pass[i].K;
    }
    return s == L;
}

cudaError_t launch_ntt(const hx_plan_s* plan, uint64_t* out, const uint64_t* in,
                       uint32_t n_polys, bool forward, uint32_t in_mf, uint32_t out_mf,
                       const NttCfg& cfg, cudaStream_t stream) {
    (void)in_mf;  // every allowed input range is inside the butterflies' lazy range
    const int L = plan->logN;
    for (int step = 0; step < cfg.npass; ++step) {
        // forward runs passes in stage order; inverse runs them backwards
        const int pi = forward ? step : cfg.npass - 1 - step;
        const PassCfg& p = cfg.pass[pi];
        PassArgs a;
        a.out = out;
        a.in = step == 0 ? in : out;
        a.limbs = plan->d_limbs;
        a.n_limbs = plan->n_limbs;
        a.n_polys = n_polys;
        a.L = L;
        a.s0 = p.s0;
        a.logGb = p.logGb;
        a.logGc = p.logGc;
        const int w = L - p.s0 - p.K;
        a.log_tiles_c = w - p.logGc;
        a.last = step == cfg.npass - 1;
        a.out_mf = out_mf;
        const int logTE = p.logGb + p.K + p.logGc;
        const uint32_t tiles = 1u << (L - logTE);
        const uint32_t threads = 1u << (logTE - p.logR);
        const size_t smem = (size_t)8 << logTE;
        PassKernel k = pick(forward, p.logR, p.K);
        if (!k) return cudaErrorInvalidConfiguration;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute((const void*)k,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        dim3 grid(tiles * n_polys, plan->n_limbs);
        k<<<grid, threads, smem, stream>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hx
