// Fused negacyclic NTT pass kernels for sm_103a (templates; instantiated in
// ntt_fwd.cu and ntt_inv.cu).
//
// The forward transform is the radix-2 Cooley-Tukey NTT of Section 2.2 with
// the Harvey butterfly (values kept lazily in [0, 2m)); the inverse is the
// radix-2 Gentleman-Sande InvNTT with the Harvey inverse butterfly (values in
// [0, m)) and the N^-1 scaling folded into its last stage, m = 2q with the
// exact Shoup quotient, 4q with the truncated one (Word below).  Both index the
// twiddles as the paper's algorithms do: stage s (s = 0 .. log2 N - 1,
// m = 2^s) pairs element j with j + N/2^(s+1) and uses table entry
// 2^s + (j >> (log2 N - s)) -- psi_rev for the forward, psi^-1_rev for the
// inverse, whose loop runs the same stages in reverse order.
//
// GPU design (not the paper's AVX512 one): a pass takes K consecutive stages
// for a tile of 2^logGb x 2^K x 2^logGc elements that those stages keep
// closed (fixed top index bits b, fixed low index bits c).  Within the tile
// the K stages run as register rounds: each thread holds 2^LOG_R elements and
// applies up to LOG_R stages to them entirely in registers; consecutive
// rounds exchange through an XOR-swizzled shared-memory tile.  The first
// round reads its registers straight from HBM and the last round writes
// straight back whenever the round's element-to-thread map is coalesced
// (column passes, and the low-stage end of row passes); otherwise the tile is
// staged through shared memory with 16-byte vector copies.  Twiddle pairs
// {W, W'} are read through the read-only path from one base pointer per
// (round, sub-stage, group) plus compile-time offsets, or from a copy of the
// tile's pairs staged in shared memory.  A persistent double-buffered
// variant streams tiles with cp.async.
#pragma once
#include <stdint.h>

#include "hx_internal.h"
#include "modarith.cuh"

namespace hx {

struct PassArgs {
    uint64_t* out;
    const uint64_t* in;
    const LimbDev* limbs;
    const uint32_t* order;   // grid row -> limb (the plan's launch order), or nullptr: row = limb
    uint32_t n_limbs;
    uint32_t n_polys;
    int L;            // log2 N
    int s0;           // first stage of the pass
    int logGb;        // log2 of top-index values per tile
    int logGc;        // log2 of low-index values per tile (0 when the pass ends at stage L-1)
    int log_tiles_c;  // log2 of tiles along the low index
    uint32_t last;    // this pass finishes the transform
    uint32_t out_mf;  // output mod factor (applied when last)
};

// K stages split into ceil(K / LOG_R) rounds of near-equal size; round i
// covers e-bits [off(i), off(i) + size(i)) counted from the top (the pass's
// first stage acts on the top e-bit).
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

// Shared-memory position of local element l in the per-tile kernels: one pad
// word after every 16, so column-wise and stride-2^r row-wise half-warp
// accesses hit distinct 8-byte bank pairs.  For a register offset v << s
// (disjoint from the group's base bits) the position is
// pad(base) + (v << s) + ((v << s) >> 4): a compile-time constant whenever s
// is, so those accesses need no address arithmetic.
__device__ __forceinline__ uint32_t pad(uint32_t l) { return l + (l >> 4); }
__host__ __device__ constexpr uint32_t padded(uint32_t te) { return te + (te >> 4); }
__device__ __forceinline__ uint32_t pad_off(uint32_t v, int s) { return (v << s) + ((v << s) >> 4); }

// Word<Wd, AR>: butterflies on Wd-sized words.  AR = 0 uses the exact Shoup
// product (lazy bound m = 2q: forward values in [0, 4q), inverse in [0, 2q),
// the paper's ranges); AR = 1 (64-bit words, q < 2^61) uses the truncated
// quotient, whose product lies in [0, 4q), so m = 4q: forward values in
// [0, 8q), inverse in [0, 4q).  Either way every output is w x mod q
// exactly; only the lazy representative differs.
template <typename Wd, int AR = 0>
struct Word;

template <int AR>
struct Word<uint64_t, AR> {
    static constexpr int V = AR ? 3 : HX_SHOUP_VARIANT;
    static constexpr uint32_t M = AR ? 4 : 2;
    static __device__ __forceinline__ void fwd(uint64_t& a, uint64_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t m) {
        harvey_fwd64<V>(a, b, w.x, w.y, q, m);
    }
    static __device__ __forceinline__ void inv(uint64_t& a, uint64_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t m) {
        harvey_inv64<V>(a, b, w.x, w.y, q, m);
    }
    static __device__ __forceinline__ uint64_t mul(uint64_t x, uint64_t w, uint64_t wp,
                                                   uint64_t q) {
        return shoup_lazy64v<V>(x, w, wp, q, 0 - q);
    }
};

template <>
struct Word<uint32_t, 0> {
    static constexpr uint32_t M = 2;
    static __device__ __forceinline__ void fwd(uint32_t& a, uint32_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t m) {
        harvey_fwd32(a, b, (uint32_t)w.x, (uint32_t)w.y, (uint32_t)q, (uint32_t)m);
    }
    static __device__ __forceinline__ void inv(uint32_t& a, uint32_t& b, ulonglong2 w, uint64_t q,
                                               uint64_t m) {
        harvey_inv32(a, b, (uint32_t)w.x, (uint32_t)w.y, (uint32_t)q, (uint32_t)m);
    }
    static __device__ __forceinline__ uint32_t mul(uint32_t x, uint64_t w, uint64_t wp,
                                                   uint64_t q) {
        return shoup_mul_lazy32(x, (uint32_t)w, (uint32_t)wp, (uint32_t)q);
    }
};

// Final correction of a transform's last stage: values in [0, B q) (B = 2m/q
// for the forward, m/q for the inverse) brought into [0, out_mf q) by
// conditional subtractions of (B/2) q, (B/4) q, ..., out_mf q.
template <typename Wd, int B>
__device__ __forceinline__ Wd to_out_range(Wd y, uint64_t q, uint32_t out_mf) {
#pragma unroll
    for (int k = B / 2; k >= 1; k >>= 1) {
        if (out_mf <= (uint32_t)k) {
            const Wd kq = (Wd)((uint64_t)k * q);
            y = y >= kq ? y - kq : y;
        }
    }
    return y;
}

// 16-byte asynchronous copies global -> shared (cp.async, bypassing registers).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct TileCtx {
    const uint64_t* gin;   // this transform's input, element 0
    uint64_t* gout;        // this transform's output, element 0
    uint64_t b_base;       // first top-index value of the tile
    uint64_t c_base;       // first low-index value of the tile
    int L, s0, logGc, w;   // w = L - s0 - K: low bits below the pass's stages
    int logGb = 0;         // log2 of top-index values per tile
    uint32_t nthreads;
    uint32_t out_mf;
    bool last;
    uint64_t poly_stride = 0;   // elements between the same limb of consecutive polynomials
    uint32_t np_valid = 1;      // polynomials of this block's group that exist
    // Cluster-fused transforms (ntt_cluster.cuh): the round that reads its
    // elements from the other phase's layout in the cluster's shared memory.
    const uint64_t* gin2 = nullptr;   // dyadic product: the second operand (see tile_mul_to_smem)
    uint32_t mul_mf = 4;              // ... and the input range factor of both operands
    uint32_t xsm = 0;      // shared-window address of this CTA's data tile
    int xK2 = 0;           // row-phase stages (log2 of a row's length)
    int xlogGc = 0;        // log2 of the columns each CTA holds in the column phase
    int xlogGb = 0;        // log2 of the rows each CTA holds in the row phase
};

// Global index of local tile element l = (bl, e, cl).  Row passes (ROW: the
// pass ends at the last stage, w = 0) hold whole rows, so their tile is the
// contiguous range from b_base << K.
template <int K, bool ROW = false>
__device__ __forceinline__ uint64_t tile_gidx(uint32_t l, const TileCtx& t) {
    if (ROW || t.w == 0) return (t.b_base << K) + l;
    const uint32_t cl = l & ((1u << t.logGc) - 1);
    const uint32_t rho = l >> t.logGc;
    const uint64_t e = rho & ((1u << K) - 1);
    const uint64_t bl = rho >> K;
    return ((t.b_base + bl) << (t.L - t.s0)) + (e << t.w) + t.c_base + cl;
}

enum { IO_SMEM = 0, IO_GLOBAL = 1, IO_DSMEM = 2 };

// Thread-block cluster primitives (sm_90+ PTX): the barrier every thread of
// every CTA of the cluster takes (release/acquire orders the shared-memory
// writes before it with the remote reads after it), and an 8-byte load from
// another CTA's shared memory at the same offset as `local` (a shared-window
// address of this CTA) in CTA `rank`.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint64_t ld_dsmem_u64(uint32_t local, uint32_t rank) {
    uint32_t ra;
    uint64_t x;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(local), "r"(rank));
    asm volatile("ld.shared::cluster.u64 %0, [%1];\n" : "=l"(x) : "r"(ra));
    return x;
}

// Element l of this CTA's tile in the exchange round of a cluster-fused
// transform of N = 2^K1 x 2^K2 (index = row << K2 | col; the column phase runs
// stages 0 .. K1-1 on the row bits, the row phase stages K1 .. L-1 on the
// column bits).  In the column phase CTA k holds columns
// [k 2^xlogGc, (k+1) 2^xlogGc) of every row, at local index row << xlogGc |
// col'; in the row phase rows [k 2^xlogGb, (k+1) 2^xlogGb) of every column,
// at local index row' << K2 | col.  FROM_COLUMN: l indexes a row-phase tile
// (the forward's exchange) whose data sits in the column-phase layout;
// otherwise l indexes a column-phase tile (the inverse's exchange) whose data
// sits in the row-phase layout.
template <bool FROM_COLUMN>
__device__ __forceinline__ uint64_t exchange_load(const TileCtx& c, uint32_t l) {
    uint32_t owner, rl;
    if (FROM_COLUMN) {
        const uint32_t row = (uint32_t)c.b_base + (l >> c.xK2);
        const uint32_t col = l & ((1u << c.xK2) - 1);
        owner = col >> c.xlogGc;
        rl = (row << c.xlogGc) | (col & ((1u << c.xlogGc) - 1));
    } else {
        const uint32_t row = l >> c.logGc;
        owner = row >> c.xlogGb;
        rl = ((row & ((1u << c.xlogGb) - 1)) << c.xK2) |
             ((uint32_t)c.c_base + (l & ((1u << c.logGc) - 1)));
    }
    return ld_dsmem_u64(c.xsm + 8u * pad(rl), owner);
}

// One register round: stages s0+P .. s0+P+R-1 of the pass.  Each thread holds
// 2^LOG_R elements = U = 2^(LOG_R-R) independent groups of 2^R; register index
// reg = (v << (LOG_R - R)) | u, so the butterfly pair of sub-stage k differs
// in register bit LOG_R-1-k (a compile-time position).  Group g = u * T + tid
// (T threads) has bits [bl | e_hi (P) | e_lo (K-P-R) | cl (logGc)].
// With NP > 1 the thread holds the same positions of NP polynomials (same
// limb, same twiddles): every twiddle pair it loads serves NP butterflies.
// Polynomial p's tile lives at sm + p * TE in shared memory.
// With TWS the twiddles come from the tile's staged copy in shared memory
// (stage_twiddles), `tw` pointing at it; WAIT_TW makes this round wait for
// that copy after issuing its own loads.
template <bool FWD, typename Wd, int AR, int LOG_R, int K, int P, int R, int SRC, int DST,
          int NP = 1, bool ROW = false, bool TWS = false, bool WAIT_TW = false, bool PF = false>
__device__ __forceinline__ void ntt_round(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                          const LimbDev& lc, const TileCtx& c) {
    constexpr int RN = 1 << LOG_R;
    constexpr int U = 1 << (LOG_R - R);
    constexpr int ELO = K - P - R;
    const uint32_t TEP = padded(c.nthreads << LOG_R);
    Wd xs[NP][RN];
    uint32_t hp[U];   // 2^(s0+P) + the group's prefix: sub-stage k's twiddles start at hp << k
    uint32_t lbase[U], hiu[U];
    const uint32_t cmask = (1u << c.logGc) - 1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t g = u * c.nthreads + threadIdx.x;
        const uint32_t cl = g & cmask;
        const uint32_t t1 = g >> c.logGc;
        const uint32_t elo = t1 & ((1u << ELO) - 1);
        const uint32_t t2 = t1 >> ELO;
        const uint32_t ehi = t2 & ((1u << P) - 1);
        const uint32_t bl = t2 >> P;
        lbase[u] = (bl << (K + c.logGc)) | (ehi << (K - P + c.logGc)) | (elo << c.logGc) | cl;
        hp[u] = (1u << (c.s0 + P)) | (((uint32_t)c.b_base + bl) << P) | ehi;
        hiu[u] = (bl << P) | ehi;
    }
    const int sshift = ROW ? ELO : ELO + c.logGc;   // v stride in the tile
    const int gshift = ROW ? ELO : ELO + c.w;       // v stride in global memory
    if constexpr (PF) {
        // ask L1 for the round's twiddle lines before the data arrives:
        // sub-stage k reads the 2^k pairs from entry hp << k (<= 128 bytes
        // for k <= 3, one line when aligned)
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const ulonglong2* p = tw + (hp[u] << k);
#pragma unroll
                for (int b = 0; b < ((16 << k) + 127) / 128; ++b)
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(p + 8 * b));
            }
        }
    }
    uint32_t pl[U];
#pragma unroll
    for (int u = 0; u < U; ++u) pl[u] = pad(lbase[u]);

#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
        Wd* x = xs[pp];
        if (NP > 1 && pp >= (int)c.np_valid) {   // no such polynomial: idle registers
#pragma unroll
            for (int reg = 0; reg < RN; ++reg) x[reg] = 0;
            continue;
        }
        if (SRC == IO_GLOBAL) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t* p = c.gin + pp * c.poly_stride + tile_gidx<K, ROW>(lbase[u], c);
#pragma unroll
                for (int v = 0; v < (1 << R); ++v)
                    x[(v << (LOG_R - R)) | u] = (Wd)__ldg(p + ((uint64_t)v << gshift));
            }
        } else if (SRC == IO_DSMEM) {
            // the forward's exchange is in its row phase (ROW), the inverse's
            // in its column phase
#pragma unroll
            for (int reg = 0; reg < RN; ++reg) {
                const int u = reg & (U - 1), v = reg >> (LOG_R - R);
                x[reg] = (Wd)exchange_load<ROW>(c, lbase[u] | ((uint32_t)v << sshift));
            }
        } else {
            const uint64_t* smp = sm + pp * TEP;
#pragma unroll
            for (int reg = 0; reg < RN; ++reg) {
                const int u = reg & (U - 1), v = reg >> (LOG_R - R);
                x[reg] = (Wd)smp[pl[u] + pad_off(v, sshift)];
            }
        }
    }
    if constexpr (WAIT_TW) {
        cp_async_wait<0>();
        __syncthreads();
    }

    const uint64_t q = lc.q, qm = (uint64_t)Word<Wd, AR>::M * lc.q;
#pragma unroll
    for (int kk = 0; kk < R; ++kk) {
        const int k = FWD ? kk : R - 1 - kk;   // sub-stage: stage c.s0 + P + k
        const int hb = LOG_R - 1 - k;
        if (!FWD && P == 0 && k == 0 && c.s0 == 0) {
            // stage 0 of the inverse: N^-1 folded into the last butterfly
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
                for (int reg0 = 0; reg0 < RN; ++reg0) {
                    if (reg0 & (1 << hb)) continue;
                    const int reg1 = reg0 | (1 << hb);
                    const Wd a = xs[pp][reg0], b = xs[pp][reg1];
                    const Wd sum = a + b;              // [0, 2m)
                    const Wd dif = a - b + (Wd)qm;     // (0, 2m)
                    xs[pp][reg0] = Word<Wd, AR>::mul(sum, lc.ninv, lc.ninv_p, q);
                    xs[pp][reg1] = Word<Wd, AR>::mul(dif, lc.ninv_w, lc.ninv_w_p, q);
                }
            }
            continue;
        }
        const ulonglong2* tb[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            tb[u] = TWS ? tw + ((((1u << (P + k)) - 1) << c.logGb) + hiu[u]) : tw + (hp[u] << k);
#pragma unroll
        for (int reg0 = 0; reg0 < RN; ++reg0) {
            if (reg0 & (1 << hb)) continue;
            const int reg1 = reg0 | (1 << hb);
            const int u = reg0 & (U - 1), v0 = reg0 >> (LOG_R - R);
            const ulonglong2 w = TWS ? tb[u][(uint32_t)(v0 >> (R - k)) << (c.logGb + P)]
                                     : __ldg(tb[u] + (v0 >> (R - k)));
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
                if (FWD)
                    Word<Wd, AR>::fwd(xs[pp][reg0], xs[pp][reg1], w, q, qm);
                else
                    Word<Wd, AR>::inv(xs[pp][reg0], xs[pp][reg1], w, q, qm);
            }
        }
    }
    if (c.last) {
        constexpr int B = (FWD ? 2 : 1) * Word<Wd, AR>::M;
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
            for (int reg = 0; reg < RN; ++reg)
                xs[pp][reg] = to_out_range<Wd, B>(xs[pp][reg], q, c.out_mf);
        }
    }

    // every CTA of the cluster has read what it needs from this CTA's tile
    // before this CTA overwrites it
    if constexpr (SRC == IO_DSMEM) cluster_sync_all();
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
        if (NP > 1 && pp >= (int)c.np_valid) continue;
        const Wd* x = xs[pp];
        if (DST == IO_GLOBAL) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint64_t* p = c.gout + pp * c.poly_stride + tile_gidx<K, ROW>(lbase[u], c);
#pragma unroll
                for (int v = 0; v < (1 << R); ++v)
                    p[(uint64_t)v << gshift] = (uint64_t)x[(v << (LOG_R - R)) | u];
            }
        } else {
            uint64_t* smp = sm + pp * TEP;
#pragma unroll
            for (int reg = 0; reg < RN; ++reg) {
                const int u = reg & (U - 1), v = reg >> (LOG_R - R);
                smp[pl[u] + pad_off(v, sshift)] = (uint64_t)x[reg];
            }
        }
    }
}

// Cooperative coalesced copies of the whole tile (of each of the block's NP
// polynomials) between HBM and shared memory.  Only row passes stage their
// tiles, so the tile is the contiguous range from b_base << K.  Each thread
// moves 2^(LOG_R-1) pairs; the loop count is a compile-time constant so that
// all of a thread's loads are in flight before the first store.
template <int K, int LOG_R, int NP = 1>
__device__ __forceinline__ void tile_to_smem(uint64_t* sm, const TileCtx& c, uint32_t TE) {
    constexpr int IT = 1 << (LOG_R - 1);
    for (uint32_t pp = 0; pp < (NP > 1 ? c.np_valid : 1u); ++pp) {
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(
            c.gin + pp * c.poly_stride + (c.b_base << K));
        uint64_t* smp = sm + pp * padded(TE);
        ulonglong2 v[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) v[it] = __ldg(src + threadIdx.x + it * c.nthreads);
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const uint32_t l = 2 * (threadIdx.x + it * c.nthreads);
            smp[pad(l)] = v[it].x;        // l even: l and l + 1 share one 16-word row
            smp[pad(l) + 1] = v[it].y;
        }
    }
}

template <int K, int LOG_R, int NP = 1>
__device__ __forceinline__ void smem_to_tile(const uint64_t* sm, const TileCtx& c, uint32_t TE) {
    constexpr int IT = 1 << (LOG_R - 1);
    for (uint32_t pp = 0; pp < (NP > 1 ? c.np_valid : 1u); ++pp) {
        ulonglong2* dst =
            reinterpret_cast<ulonglong2*>(c.gout + pp * c.poly_stride + (c.b_base << K));
        const uint64_t* smp = sm + pp * padded(TE);
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const uint32_t i = threadIdx.x + it * c.nthreads, l = 2 * i;
            dst[i] = make_ulonglong2(smp[pad(l)], smp[pad(l) + 1]);
        }
    }
}

// The dyadic product of Listing 4 (MultMod with input_mod_factor 1, 2 or 4)
// as the staging step of the inverse's first pass: the tile of
// c_i = a_i b_i mod q in [0, q) -- EltwiseMultMod's value -- a from c.gin and
// b from c.gin2 (forward outputs below mul_mf q), written to shared memory
// where tile_to_smem would write a.  Wd: the limb's word class (mulmod_fused:
// 32-bit words below 2^30, truncated Barrett quotients below 2^61).  Both
// tiles are read with 16-byte loads; the product never goes to HBM.
template <int K, int LOG_R, int NP, int Wd>
__device__ __forceinline__ void tile_mul_to_smem(uint64_t* sm, const TileCtx& c, uint32_t TE,
                                                 const LimbDev& lc) {
    constexpr int IT = 1 << (LOG_R - 1);
    const uint64_t q = lc.q, bk = lc.barrett_k;
    const uint32_t Qm1 = lc.barrett_qm1;
    const uint32_t mf = c.mul_mf;
    for (uint32_t pp = 0; pp < (NP > 1 ? c.np_valid : 1u); ++pp) {
        const uint64_t off = pp * c.poly_stride + (c.b_base << K);
        const ulonglong2* A = reinterpret_cast<const ulonglong2*>(c.gin + off);
        const ulonglong2* B = reinterpret_cast<const ulonglong2*>(c.gin2 + off);
        uint64_t* smp = sm + pp * padded(TE);
        ulonglong2 va[IT], vb[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            va[it] = __ldg(A + threadIdx.x + it * c.nthreads);
            vb[it] = __ldg(B + threadIdx.x + it * c.nthreads);
        }
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const uint32_t l = 2 * (threadIdx.x + it * c.nthreads);
            smp[pad(l)] = mulmod_fused<Wd>(small_mod_rt(va[it].x, q, mf),
                                           small_mod_rt(vb[it].x, q, mf), q, bk, Qm1);
            smp[pad(l) + 1] = mulmod_fused<Wd>(small_mod_rt(va[it].y, q, mf),
                                               small_mod_rt(vb[it].y, q, mf), q, bk, Qm1);
        }
    }
}

// Executes round I (in execution order) and the ones after it.  COLUMN
// passes (logGc > 0) read and write HBM directly in their first and last
// rounds; row passes do so at their low-stage end only (the forward's first
// round, the inverse's last) and stage the high-stage end through shared
// memory, where the round's thread map is strided.
template <bool FWD, bool COLUMN, typename Wd, int AR, int LOG_R, int K, int I, int NP = 1,
          bool TWS = false>
__device__ __forceinline__ void ntt_rounds(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                           const LimbDev& lc, const TileCtx& c) {
    using S = Sched<K, LOG_R>;
    constexpr int NR = S::NR;
    constexpr int idx = FWD ? I : NR - 1 - I;
    constexpr bool first = I == 0, lastr = I == NR - 1;
    constexpr bool direct_in = first && (COLUMN || FWD);
    constexpr bool direct_out = lastr && (COLUMN || !FWD);
    TileCtx cr = c;
    cr.last = c.last && lastr;
    ntt_round<FWD, Wd, AR, LOG_R, K, S::off(idx), S::size(idx), direct_in ? IO_GLOBAL : IO_SMEM,
              direct_out ? IO_GLOBAL : IO_SMEM, NP, !COLUMN, TWS, TWS && direct_in>(sm, tw, lc,
                                                                                 cr);
    if constexpr (!lastr) {
        __syncthreads();
        ntt_rounds<FWD, COLUMN, Wd, AR, LOG_R, K, I + 1, NP, TWS>(sm, tw, lc, c);
    }
}

// Copies the twiddle pairs of every stage of the tile into shared memory
// (asynchronously; the caller commits and waits).  Stage p of the pass uses
// table entries 2^(s0+p) + (b << p) + e for the tile's 2^logGb top-index
// values b and e < 2^p: 2^(logGb+p) consecutive pairs, stored from
// 2^logGb (2^p - 1) on.  Within a stage, entry i = (h << k) + j -- k the
// stage's position in its register round (round offset P), h = (b_local << P)
// | e_hi the group's index -- goes to (j << (logGb + P)) + h, so that for
// each j the groups of consecutive threads read consecutive pairs.
template <int K, int LOG_R>
__device__ __forceinline__ void stage_twiddles(ulonglong2* tws, const ulonglong2* __restrict__ tw,
                                               const TileCtx& c) {
    using S = Sched<K, LOG_R>;
    const int lgb = c.logGb;
#pragma unroll
    for (int p = 0; p < K; ++p) {
        int P = 0;
#pragma unroll
        for (int r = 0; r < S::NR; ++r)
            if (p >= S::off(r)) P = S::off(r);
        const int k = p - P;
        const uint32_t cnt = 1u << (lgb + p);
        const ulonglong2* src = tw + ((1ull << (c.s0 + p)) + (c.b_base << p));
        ulonglong2* dst = tws + (((1u << p) - 1) << lgb);
        for (uint32_t i = threadIdx.x; i < cnt; i += c.nthreads)
            cp_async16(dst + ((i & ((1u << k) - 1)) << (lgb + P)) + (i >> k), src + i);
    }
}

// Pairs in a tile's staged twiddle copy: 2^logGb (2^K - 1).
__host__ __device__ constexpr uint32_t staged_twiddles(int logGb, int K) {
    return ((1u << K) - 1) << logGb;
}

// The rounds of one tile for the block's NP polynomials.  A staged row pass
// of the inverse (its tiles already in shared memory) transforms them one
// after another when HX_INV_NP_SEQ is set: each polynomial's elements then
// fit the registers of one (the second polynomial's twiddle loads hit L1),
// where transforming them together shares every twiddle load but holds NP
// times the elements.
#ifndef HX_INV_NP_SEQ
#define HX_INV_NP_SEQ 1
#endif
template <bool FWD, bool COLUMN, typename Wd, int AR, int LOG_R, int K, int NP, bool TWS>
__device__ __forceinline__ void pass_rounds(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                            const LimbDev& lc, const TileCtx& c, uint32_t TE) {
    if constexpr (!FWD && !COLUMN && NP > 1 && HX_INV_NP_SEQ) {
        TileCtx cp = c;
        cp.np_valid = 1;
        const uint32_t n = c.np_valid, step = padded(TE);
#pragma unroll 1
        for (uint32_t pp = 0; pp < n; ++pp) {
            ntt_rounds<FWD, COLUMN, Wd, AR, LOG_R, K, 0, 1, TWS>(sm + pp * step, tw, lc, cp);
            cp.gout += cp.poly_stride;
        }
    } else {
        ntt_rounds<FWD, COLUMN, Wd, AR, LOG_R, K, 0, NP, TWS>(sm, tw, lc, c);
    }
}

// One tile of one pass (for each of NP polynomials), by the whole block
// (TE >> LOG_R threads): stage in through shared memory where the first
// round's map is strided, run the rounds, stage out where the last round's
// map is strided.
// With TWS the tile's twiddles are first copied to shared memory after the
// NP data tiles (stage_twiddles), overlapping the first data loads.
template <bool FWD, bool COLUMN, int LOG_R, int K, int NP = 1, bool TWS = false,
          bool MUL = false>
__device__ __forceinline__ void process_tile(uint64_t* sm, const TileCtx& c, const LimbDev& lc,
                                             uint32_t TE) {
    constexpr bool staged_in = !COLUMN && !FWD;
    constexpr bool staged_out = !COLUMN && FWD;
    const ulonglong2* tw = FWD ? lc.fwd : lc.inv;
    if constexpr (TWS) {
        ulonglong2* tws = reinterpret_cast<ulonglong2*>(sm + NP * padded(TE));
        stage_twiddles<K, LOG_R>(tws, tw, c);
        cp_async_commit();
        tw = tws;
    }
    static_assert(!MUL || staged_in, "the product stages an inverse row tile");
    if (staged_in) {
        if constexpr (MUL) {
            if (lc.narrow)
                tile_mul_to_smem<K, LOG_R, NP, 0>(sm, c, TE, lc);
            else if (lc.trunc)
                tile_mul_to_smem<K, LOG_R, NP, 1>(sm, c, TE, lc);
            else
                tile_mul_to_smem<K, LOG_R, NP, 2>(sm, c, TE, lc);
        } else
            tile_to_smem<K, LOG_R, NP>(sm, c, TE);
        if constexpr (TWS) cp_async_wait<0>();
        __syncthreads();
    }
    if (lc.narrow)
        pass_rounds<FWD, COLUMN, uint32_t, 0, LOG_R, K, NP, TWS>(sm, tw, lc, c, TE);
    else if (lc.trunc)
        pass_rounds<FWD, COLUMN, uint64_t, 1, LOG_R, K, NP, TWS>(sm, tw, lc, c, TE);
    else
        pass_rounds<FWD, COLUMN, uint64_t, 0, LOG_R, K, NP, TWS>(sm, tw, lc, c, TE);
    if (staged_out) {
        __syncthreads();
        smem_to_tile<K, LOG_R, NP>(sm, c, TE);
    }
}

// Register caps of the per-tile kernels, chosen by measurement on GB300 at
// N = 2^16 x 32 limbs (the compiler's own choice leaves fewer blocks resident
// than the latency of the loads needs): 72 with 16 elements a thread (it
// would take up to 102: forward call 104 -> 92 us under the schedule with a
// 7-stage column pass); with 8, 40 in the forward (92 -> 90 us) and 48 in
// the inverse (80 -> 74 us); 96 with two polynomials a thread in the forward
// (spills stay within 16 bytes); HX_INV_NP_MAXNREG with two in the
// inverse's row passes, which transform them one after another
// (pass_rounds).  Blocks have at
// most 512 threads, which 512 x 96 registers fit.
#ifndef HX_INV_NP_MAXNREG
#define HX_INV_NP_MAXNREG 64
#endif
#define HX_PASS_MAXNREG                                                                     \
    __maxnreg__(LOG_R == 4 ? 72                                                             \
                : NP > 1   ? (FWD || COLUMN || !HX_INV_NP_SEQ ? 96 : HX_INV_NP_MAXNREG) \
                : FWD      ? 40                                                             \
                           : 48)
// The product's staging step holds both operands' pairs: 56 with 8 elements
// a thread (no spills); with two polynomials a thread (staged one at a time,
// transformed one after another) as the inverse's row passes.
#define HX_MUL_MAXNREG __maxnreg__(LOG_R == 4 ? 72 : NP > 1 ? HX_INV_NP_MAXNREG : 56)

// One tile of one pass for each of the block's NP polynomials: block
// (tile, group of NP polynomials, limb).  MUL: the inverse's first pass
// with the dyadic product computed in its staging step.
template <bool FWD, bool COLUMN, int LOG_R, int K, int NP, bool TWS, bool MUL>
__device__ __forceinline__ void ntt_pass_body(const PassArgs& a, const uint64_t* b,
                                              uint32_t in_mf) {
    extern __shared__ uint64_t sm[];
    const uint32_t limb = a.order ? a.order[blockIdx.y] : blockIdx.y;
    const uint32_t n_groups = (a.n_polys + NP - 1) / NP;
    const uint32_t poly = (blockIdx.x % n_groups) * NP;
    const uint32_t tile = blockIdx.x / n_groups;
    const LimbDev lc = a.limbs[limb];
    const uint64_t base = ((uint64_t)poly * a.n_limbs + limb) << a.L;
    const uint32_t tile_c = tile & ((1u << a.log_tiles_c) - 1);
    const uint32_t tile_b = tile >> a.log_tiles_c;
    const uint32_t TE = 1u << (a.logGb + K + a.logGc);
    TileCtx c;
    c.gin = a.in + base;
    c.gout = a.out + base;
    c.b_base = (uint64_t)tile_b << a.logGb;
    c.c_base = (uint64_t)tile_c << a.logGc;
    c.L = a.L;
    c.s0 = a.s0;
    c.logGc = a.logGc;
    c.logGb = a.logGb;
    c.w = a.L - a.s0 - K;
    c.nthreads = TE >> LOG_R;
    c.out_mf = a.out_mf;
    c.last = a.last != 0;
    c.poly_stride = (uint64_t)a.n_limbs << a.L;
    c.np_valid = min((uint32_t)NP, a.n_polys - poly);
    if constexpr (MUL) {
        c.gin2 = b + base;
        c.mul_mf = in_mf;
    }
    process_tile<FWD, COLUMN, LOG_R, K, NP, TWS, MUL>(sm, c, lc, TE);
}

// One block per (tile, group of NP polynomials, limb).
template <bool FWD, bool COLUMN, int LOG_R, int K, int NP = 1, bool TWS = false>
__global__ void HX_PASS_MAXNREG ntt_pass_kernel(PassArgs a) {
    ntt_pass_body<FWD, COLUMN, LOG_R, K, NP, TWS, false>(a, nullptr, 4);
}

// The inverse's first (row) pass with the dyadic product of a.in and b
// (both below in_mf q) computed in its staging step (tile_mul_to_smem).
template <int LOG_R, int K, int NP, bool TWS>
__global__ void HX_MUL_MAXNREG ntt_mul_inv_kernel(PassArgs a, const uint64_t* b,
                                                  uint32_t in_mf) {
    ntt_pass_body<false, false, LOG_R, K, NP, TWS, true>(a, b, in_mf);
}


// ---------------------------------------------------------------------------
// Persistent, double-buffered variant.  Each block walks the tiles t =
// blockIdx.x, blockIdx.x + gridDim.x, ...; while it transforms tile t out of
// one shared-memory buffer, the next tile streams into the other buffer with
// cp.async (16-byte asynchronous copies that bypass the registers), so HBM
// latency hides behind the butterflies even at two blocks per SM; the next
// tile's twiddle lines are requested into L1 at the same time.
// Tiles are numbered (limb, tile, polynomial) with the polynomial fastest, so
// blocks that run together share one limb's twiddles in L1/L2.
// ---------------------------------------------------------------------------

// 16-byte-granular swizzle (keeps the two words of each aligned pair together
// so cp.async can write it): XOR bits 1..3 with bits 4..6; every round of the
// schedules used here sees at most 2-way bank conflicts.
__device__ __forceinline__ uint32_t swz16(uint32_t l) { return l ^ (((l >> 4) & 7u) << 1); }


struct TileId {
    uint32_t limb, poly, tile;
};

__device__ __forceinline__ TileId decode_tile(uint32_t t, const PassArgs& a, uint32_t tiles) {
    TileId id;
    id.poly = t % a.n_polys;
    const uint32_t r = t / a.n_polys;
    id.tile = r % tiles;
    id.limb = r / tiles;
    return id;
}

template <int K>
__device__ __forceinline__ void tile_ctx(const TileId& id, const PassArgs& a, TileCtx& c) {
    const uint64_t base = ((uint64_t)id.poly * a.n_limbs + id.limb) << a.L;
    const uint32_t tile_c = id.tile & ((1u << a.log_tiles_c) - 1);
    const uint32_t tile_b = id.tile >> a.log_tiles_c;
    c.gin = a.in + base;
    c.gout = a.out + base;
    c.b_base = (uint64_t)tile_b << a.logGb;
    c.c_base = (uint64_t)tile_c << a.logGc;
    c.L = a.L;
    c.s0 = a.s0;
    c.logGc = a.logGc;
    c.logGb = a.logGb;
    c.w = a.L - a.s0 - K;
    c.out_mf = a.out_mf;
    c.last = a.last != 0;
}

template <int K>
__device__ __forceinline__ void tile_prefetch(uint64_t* dst, const TileCtx& c, uint32_t TE) {
    for (uint32_t i = threadIdx.x; i < TE / 2; i += c.nthreads) {
        const uint32_t l = 2 * i;
        cp_async16(dst + swz16(l), c.gin + tile_gidx<K>(l, c));
    }
}

// Asks L1 for the 128-byte lines of the twiddle pairs a tile will read (stage
// p of the pass: 2^(logGb+p) pairs from entry 2^(s0+p) + (b << p)), so that
// the tile's rounds find them there.
template <int K>
__device__ __forceinline__ void twiddle_prefetch_l1(const ulonglong2* tw, const TileCtx& c) {
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const ulonglong2* src = tw + ((1ull << (c.s0 + p)) + (c.b_base << p));
        const uint32_t cnt = 1u << (c.logGb + p);
        for (uint32_t i = threadIdx.x * 8; i < cnt; i += c.nthreads * 8)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(src + i));
    }
}

template <int K>
__device__ __forceinline__ void smem16_to_tile(const uint64_t* sm, const TileCtx& c, uint32_t TE) {
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(c.gout);
    for (uint32_t i = threadIdx.x; i < TE / 2; i += c.nthreads) {
        const uint32_t l = 2 * i;
        dst[tile_gidx<K>(l, c) >> 1] = *reinterpret_cast<const ulonglong2*>(sm + swz16(l));
    }
}

// One register round of the pipelined kernel: reads its elements from the
// (swz16) tile in shared memory, writes them back there or, in the last
// round of a coalesced end, straight to HBM.
template <bool FWD, typename Wd, int AR, int LOG_R, int K, int P, int R, bool TO_GLOBAL>
__device__ __forceinline__ void pipe_round(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                           const LimbDev& lc, const TileCtx& c) {
    constexpr int RN = 1 << LOG_R;
    constexpr int U = 1 << (LOG_R - R);
    constexpr int ELO = K - P - R;
    Wd x[RN];
    uint32_t hp[U];
    uint32_t lbase[U];
    const uint32_t cmask = (1u << c.logGc) - 1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t g = u * c.nthreads + threadIdx.x;
        const uint32_t cl = g & cmask;
        const uint32_t t1 = g >> c.logGc;
        const uint32_t elo = t1 & ((1u << ELO) - 1);
        const uint32_t t2 = t1 >> ELO;
        const uint32_t ehi = t2 & ((1u << P) - 1);
        const uint32_t bl = t2 >> P;
        lbase[u] = (bl << (K + c.logGc)) | (ehi << (K - P + c.logGc)) | (elo << c.logGc) | cl;
        hp[u] = (1u << (c.s0 + P)) | (((uint32_t)c.b_base + bl) << P) | ehi;
    }
    const int sshift = ELO + c.logGc;
#pragma unroll
    for (int reg = 0; reg < RN; ++reg) {
        const int u = reg & (U - 1), v = reg >> (LOG_R - R);
        x[reg] = (Wd)sm[swz16(lbase[u] + ((uint32_t)v << sshift))];
    }

    const uint64_t q = lc.q, qm = (uint64_t)Word<Wd, AR>::M * lc.q;
#pragma unroll
    for (int kk = 0; kk < R; ++kk) {
        const int k = FWD ? kk : R - 1 - kk;
        const int hb = LOG_R - 1 - k;
        if (!FWD && P == 0 && k == 0 && c.s0 == 0) {
#pragma unroll
            for (int reg0 = 0; reg0 < RN; ++reg0) {
                if (reg0 & (1 << hb)) continue;
                const int reg1 = reg0 | (1 << hb);
                const Wd a = x[reg0], b = x[reg1];
                const Wd sum = a + b;
                const Wd dif = a - b + (Wd)qm;
                x[reg0] = Word<Wd, AR>::mul(sum, lc.ninv, lc.ninv_p, q);
                x[reg1] = Word<Wd, AR>::mul(dif, lc.ninv_w, lc.ninv_w_p, q);
            }
            continue;
        }
        const ulonglong2* tb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) tb[u] = tw + (hp[u] << k);
#pragma unroll
        for (int reg0 = 0; reg0 < RN; ++reg0) {
            if (reg0 & (1 << hb)) continue;
            const int reg1 = reg0 | (1 << hb);
            const int u = reg0 & (U - 1), v0 = reg0 >> (LOG_R - R);
            const ulonglong2 w = __ldg(tb[u] + (v0 >> (R - k)));
            if (FWD)
                Word<Wd, AR>::fwd(x[reg0], x[reg1], w, q, qm);
            else
                Word<Wd, AR>::inv(x[reg0], x[reg1], w, q, qm);
        }
    }
    if (c.last) {
        constexpr int B = (FWD ? 2 : 1) * Word<Wd, AR>::M;
#pragma unroll
        for (int reg = 0; reg < RN; ++reg) x[reg] = to_out_range<Wd, B>(x[reg], q, c.out_mf);
    }
    if (TO_GLOBAL) {
        const int gshift = ELO + c.w;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint64_t* p = c.gout + tile_gidx<K>(lbase[u], c);
#pragma unroll
            for (int v = 0; v < (1 << R); ++v)
                p[(uint64_t)v << gshift] = (uint64_t)x[(v << (LOG_R - R)) | u];
        }
    } else {
#pragma unroll
        for (int reg = 0; reg < RN; ++reg) {
            const int u = reg & (U - 1), v = reg >> (LOG_R - R);
            sm[swz16(lbase[u] + ((uint32_t)v << sshift))] = (uint64_t)x[reg];
        }
    }
}

template <bool FWD, bool COLUMN, typename Wd, int AR, int LOG_R, int K, int I>
__device__ __forceinline__ void pipe_rounds(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                            const LimbDev& lc, const TileCtx& c) {
    using S = Sched<K, LOG_R>;
    constexpr int NR = S::NR;
    constexpr int idx = FWD ? I : NR - 1 - I;
    constexpr bool lastr = I == NR - 1;
    TileCtx cr = c;
    cr.last = c.last && lastr;
    pipe_round<FWD, Wd, AR, LOG_R, K, S::off(idx), S::size(idx), lastr && (COLUMN || !FWD)>(
        sm, tw, lc, cr);
    if constexpr (!lastr) {
        __syncthreads();
        pipe_rounds<FWD, COLUMN, Wd, AR, LOG_R, K, I + 1>(sm, tw, lc, c);
    }
}

template <bool FWD, bool COLUMN, int LOG_R, int K>
__global__ void __maxnreg__(LOG_R == 4 ? 72 : FWD ? 40 : 48) ntt_pipe_kernel(PassArgs a) {
    extern __shared__ uint64_t sm[];
    const int logTE = a.logGb + K + a.logGc;
    const uint32_t TE = 1u << logTE;
    const uint32_t tiles = 1u << (a.L - logTE);
    const uint32_t total = tiles * a.n_polys * a.n_limbs;
    uint32_t t = blockIdx.x;
    if (t >= total) return;
    TileCtx c;
    c.nthreads = TE >> LOG_R;
    tile_ctx<K>(decode_tile(t, a, tiles), a, c);
    tile_prefetch<K>(sm, c, TE);
    cp_async_commit();
    for (uint32_t i = 0; t < total; ++i, t += gridDim.x) {
        uint64_t* buf = sm + (i & 1) * TE;
        const uint32_t tn = t + gridDim.x;
        if (tn < total) {
            TileCtx cn;
            cn.nthreads = c.nthreads;
            const TileId idn = decode_tile(tn, a, tiles);
            tile_ctx<K>(idn, a, cn);
            tile_prefetch<K>(sm + ((i + 1) & 1) * TE, cn, TE);
            twiddle_prefetch_l1<K>(FWD ? a.limbs[idn.limb].fwd : a.limbs[idn.limb].inv, cn);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const TileId id = decode_tile(t, a, tiles);
        tile_ctx<K>(id, a, c);
        const LimbDev lc = a.limbs[id.limb];
        const ulonglong2* tw = FWD ? lc.fwd : lc.inv;
        if (lc.narrow)
            pipe_rounds<FWD, COLUMN, uint32_t, 0, LOG_R, K, 0>(buf, tw, lc, c);
        else if (lc.trunc)
            pipe_rounds<FWD, COLUMN, uint64_t, 1, LOG_R, K, 0>(buf, tw, lc, c);
        else
            pipe_rounds<FWD, COLUMN, uint64_t, 0, LOG_R, K, 0>(buf, tw, lc, c);
        if (!COLUMN && FWD) {
            __syncthreads();
            smem16_to_tile<K>(buf, c, TE);
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

typedef void (*PassKernel)(PassArgs);
typedef void (*MulPassKernel)(PassArgs, const uint64_t*, uint32_t);

// ntt_mul.cu / ntt_muls.cu: the inverse's first pass with the dyadic product
// fused in, twiddles through the read-only cache / staged (nullptr: not in
// the menu)
MulPassKernel pick_mul_inv(int logR, int K, int np, bool tws);
MulPassKernel pick_mul_inv_tws(int logR, int K, int np);
// ntt_ctrow.cu: the product's step kernel (the forward's row stages on a and
// b, the dyadic product, the inverse's row stages), 8 elements a thread, 6..9
// stages; nullptr otherwise.
PassKernel pick_mul_row(int logR, int K);

// ntt_fwd.cu / ntt_inv.cu
// ntt_f1.cu, ntt_f2.cu, ntt_i1.cu, ntt_i2.cu: plain kernels with 1 or 2
// polynomials per thread, and the persistent kernels (nullptr: not in the menu)
PassKernel pick_plain_f1(bool column, int logR, int K);
PassKernel pick_plain_f2(bool column, int logR, int K);
PassKernel pick_plain_i1(bool column, int logR, int K);
PassKernel pick_plain_i2(bool column, int logR, int K);
PassKernel pick_pipe_f(bool column, int logR, int K);
PassKernel pick_pipe_i(bool column, int logR, int K);
// ntt_f1s.cu, ntt_f2s.cu, ntt_i1s.cu, ntt_i2s.cu: plain kernels with staged twiddles
PassKernel pick_tws_f1(bool column, int logR, int K);
PassKernel pick_tws_f2(bool column, int logR, int K);
PassKernel pick_tws_i1(bool column, int logR, int K);
PassKernel pick_tws_i2(bool column, int logR, int K);

}  // namespace hx
