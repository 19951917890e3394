// Cluster-fused negacyclic NTT: one thread-block cluster per limb-transform,
// every stage in on-chip memory, each coefficient read from and written to
// HBM once.
//
// The transform of N = 2^K1 x 2^K2 points (index = row << K2 | col) splits
// into the K1 stages on the row bits (Algorithm CT's first stages, Algorithm
// GS's last: the "column phase", independent 2^K1-point transforms down each
// column) and the K2 stages on the column bits (the "row phase", independent
// 2^K2-point transforms along each row with row-dependent twiddles).  A
// cluster of C = 2^LOG_C CTAs holds the limb's N coefficients in its shared
// memory, N / C per CTA:
//   column phase: CTA k holds columns [k 2^logGc, (k+1) 2^logGc) of every
//                 row (logGc = K2 - LOG_C) -- the tile of a column pass of
//                 the two-pass schedule;
//   row phase:    CTA k holds rows [k 2^logGb, (k+1) 2^logGb) of every column
//                 (logGb = K1 - LOG_C) -- the tile of a row pass.
// Both phases run the register rounds of ntt_kernels.cuh on their tile.
// Between them one round reads its elements straight from the other CTAs'
// shared memory (distributed shared memory, ld.shared::cluster), transforms
// them in registers, waits at a cluster barrier until every CTA has read its
// share, and only then overwrites its own tile.  The second HBM round trip of
// the two-pass schedule (and its load latency) disappears: one coalesced HBM
// read at the start, one write at the end.
//
// Forward: column phase first (its first round reads the column tile from
// HBM), exchange into the row phase, whose last round goes out through shared
// memory with 16-byte stores.  Inverse: row phase first (the tile is staged in
// with 16-byte loads, or computed there from the ciphertext-tensor operands),
// exchange into the column phase, whose last round (stage 0, N^-1 folded in)
// writes the columns to HBM.
//
// Every CTA of a cluster executes the same two cluster barriers and touches
// other CTAs' shared memory only between them, so no CTA exits or
// overwrites its tile while another still reads it.
#pragma once
#include "ntt_kernels.cuh"
#include "ntt_tensor.h"

namespace hx {

// Row-phase rounds ask L1 for their twiddle lines first (the row phase's
// twiddles depend on the row, so they come from L2; the column phase's are
// shared by the whole tile).
#ifndef HX_CLUSTER_PF
#define HX_CLUSTER_PF 1
#endif

// Executes round I (in execution order) of a phase and the ones after it:
// the first reads from FIRST (HBM, shared memory, or the exchange), the last
// writes to LAST; every other round goes through this CTA's shared memory.
template <bool FWD, bool COLUMN, typename Wd, int AR, int LOG_R, int K, int I, int FIRST,
          int LAST>
__device__ __forceinline__ void cl_rounds(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                          const LimbDev& lc, const TileCtx& c) {
    using S = Sched<K, LOG_R>;
    constexpr int NR = S::NR;
    constexpr int idx = FWD ? I : NR - 1 - I;
    constexpr bool lastr = I == NR - 1;
    TileCtx cr = c;
    cr.last = c.last && lastr;
    ntt_round<FWD, Wd, AR, LOG_R, K, S::off(idx), S::size(idx), I == 0 ? FIRST : IO_SMEM,
              lastr ? LAST : IO_SMEM, 1, !COLUMN, false, false,
              HX_CLUSTER_PF != 0 && !COLUMN>(sm, tw, lc, cr);
    if constexpr (!lastr) {
        __syncthreads();
        cl_rounds<FWD, COLUMN, Wd, AR, LOG_R, K, I + 1, FIRST, LAST>(sm, tw, lc, c);
    }
}

// Both phases of one limb-transform on words Wd, from the tile already in
// place for the first phase (forward: in HBM; inverse: in shared memory).
template <bool FWD, typename Wd, int AR, int LOG_R, int K1, int K2>
__device__ __forceinline__ void cluster_phases(uint64_t* sm, const LimbDev& lc,
                                               const TileCtx& col, const TileCtx& row) {
    const ulonglong2* tw = FWD ? lc.fwd : lc.inv;
    if constexpr (FWD) {
        cl_rounds<true, true, Wd, AR, LOG_R, K1, 0, IO_GLOBAL, IO_SMEM>(sm, tw, lc, col);
        cluster_sync_all();   // column-phase tiles complete and visible cluster-wide
        cl_rounds<true, false, Wd, AR, LOG_R, K2, 0, IO_DSMEM, IO_SMEM>(sm, tw, lc, row);
    } else {
        cl_rounds<false, false, Wd, AR, LOG_R, K2, 0, IO_SMEM, IO_SMEM>(sm, tw, lc, row);
        cluster_sync_all();   // row-phase tiles complete and visible cluster-wide
        cl_rounds<false, true, Wd, AR, LOG_R, K1, 0, IO_DSMEM, IO_GLOBAL>(sm, tw, lc, col);
    }
}

template <bool FWD, int LOG_R, int K1, int K2>
__device__ __forceinline__ void cluster_dispatch(uint64_t* sm, const LimbDev& lc,
                                                 const TileCtx& col, const TileCtx& row) {
    if (lc.narrow)
        cluster_phases<FWD, uint32_t, 0, LOG_R, K1, K2>(sm, lc, col, row);
    else if (lc.trunc)
        cluster_phases<FWD, uint64_t, 1, LOG_R, K1, K2>(sm, lc, col, row);
    else
        cluster_phases<FWD, uint64_t, 0, LOG_R, K1, K2>(sm, lc, col, row);
}

// Tile contexts of this CTA (cluster rank `rank`) for both phases of the
// transform whose element 0 is at gin / gout.  a.logGc = K2 - LOG_C.
template <bool FWD, int K1, int K2>
__device__ __forceinline__ void cluster_ctx(TileCtx& col, TileCtx& row, const PassArgs& a,
                                            uint32_t rank, const uint64_t* gin, uint64_t* gout,
                                            uint64_t* sm, uint32_t nthreads) {
    const int logC = K2 - a.logGc;
    col.gin = gin;
    col.gout = gout;
    col.b_base = 0;
    col.c_base = (uint64_t)rank << a.logGc;
    col.L = K1 + K2;
    col.s0 = 0;
    col.logGc = a.logGc;
    col.logGb = 0;
    col.w = K2;
    col.nthreads = nthreads;
    col.out_mf = a.out_mf;
    col.last = !FWD;   // the inverse ends in the column phase, the forward in the row phase
    col.xsm = (uint32_t)__cvta_generic_to_shared(sm);
    col.xK2 = K2;
    col.xlogGc = a.logGc;
    col.xlogGb = K1 - logC;
    row = col;
    row.c_base = 0;
    row.b_base = (uint64_t)rank << (K1 - logC);
    row.s0 = K1;
    row.logGc = 0;
    row.logGb = K1 - logC;
    row.w = 0;
    row.last = FWD;
}

// Register cap: two 512-thread CTAs (or one of 1024) per SM.
#define HX_CLUSTER_MAXNREG __maxnreg__(64)

// One cluster of 2^LOG_C CTAs per (polynomial, limb); grid (2^LOG_C n_polys,
// limbs), cluster (2^LOG_C, 1, 1); limbs in the plan's launch order.
template <bool FWD, int LOG_R, int K1, int K2>
__global__ void HX_CLUSTER_MAXNREG ntt_cluster_kernel(PassArgs a) {
    extern __shared__ uint64_t sm[];
    const int logC = K2 - a.logGc;
    const uint32_t rank = cluster_ctarank();
    const uint32_t poly = blockIdx.x >> logC;
    const uint32_t limb = a.order ? a.order[blockIdx.y] : blockIdx.y;
    const LimbDev lc = a.limbs[limb];
    const uint64_t base = ((uint64_t)poly * a.n_limbs + limb) << (K1 + K2);
    const uint32_t E = 1u << (K1 + K2 - logC);
    TileCtx col, row;
    cluster_ctx<FWD, K1, K2>(col, row, a, rank, a.in + base, a.out + base, sm, E >> LOG_R);
    if constexpr (!FWD) {
        tile_to_smem<K2, LOG_R>(sm, row, E);
        __syncthreads();
    }
    cluster_dispatch<FWD, LOG_R, K1, K2>(sm, lc, col, row);
    if constexpr (FWD) {
        __syncthreads();
        smem_to_tile<K2, LOG_R>(sm, row, E);
    }
}

// The CTA's row-phase tile of r_k into shared memory, two elements per
// step; Wd: the limb's word class (tensor_rk).
template <int Wd, int LOG_R>
__device__ __forceinline__ void cluster_tensor_tile(uint64_t* sm, const TensorIn& t,
                                                    const TensorK& tk, uint64_t base, uint64_t S,
                                                    uint32_t k, uint32_t nthreads) {
    const ulonglong2* A0 = reinterpret_cast<const ulonglong2*>(t.A + base);
    const ulonglong2* A1 = reinterpret_cast<const ulonglong2*>(t.A + S + base);
    const ulonglong2* B0 = reinterpret_cast<const ulonglong2*>(t.A + 2 * S + base);
    const ulonglong2* B1 = reinterpret_cast<const ulonglong2*>(t.A + 3 * S + base);
    const ulonglong2* Ek = reinterpret_cast<const ulonglong2*>(t.E + k * S + base);
    const ulonglong2 zero = make_ulonglong2(0, 0);
    const bool need0 = k != 2, need1 = k != 0;
#pragma unroll 4
    for (int it = 0; it < (1 << (LOG_R - 1)); ++it) {
        const uint32_t i = threadIdx.x + it * nthreads;
        const uint32_t l = 2 * i;   // l even: l and l + 1 share one 16-word row
        const ulonglong2 x0 = need0 ? __ldg(A0 + i) : zero;
        const ulonglong2 x1 = need1 ? __ldg(A1 + i) : zero;
        const ulonglong2 y0 = need0 ? __ldg(B0 + i) : zero;
        const ulonglong2 y1 = need1 ? __ldg(B1 + i) : zero;
        const ulonglong2 e = __ldg(Ek + i);
        sm[pad(l)] = tensor_rk<Wd>(k, x0.x, x1.x, y0.x, y1.x, e.x, tk);
        sm[pad(l) + 1] = tensor_rk<Wd>(k, x0.y, x1.y, y0.y, y1.y, e.y, tk);
    }
}

// The ciphertext tensor fused into the cluster inverse: the row-phase tile of
// output k is computed in shared memory from the forward outputs A0, A1, B0,
// B1 (< in_mf q) and the addend e_k (< q), r_k = (d_k s + e_k) mod q with d0 =
// A0 B0, d1 = A0 B1 + A1 B0, d2 = A1 B1 (the element-wise tensor kernel's
// values, tensor_rk's arithmetic), then inverse-transformed.  Grid (2^LOG_C 3 n_ct, limbs of
// the launch): cluster index = 3 ct + k, so the three outputs of one
// ciphertext run side by side and share the operands through L2.
template <int LOG_R, int K1, int K2>
__global__ void HX_CLUSTER_MAXNREG ntt_cluster_tensor_kernel(PassArgs a, TensorIn t) {
    extern __shared__ uint64_t sm[];
    const int logC = K2 - a.logGc;
    const uint32_t rank = cluster_ctarank();
    const uint32_t ci = blockIdx.x >> logC;
    const uint32_t k = ci % 3, p = ci / 3;
    const uint32_t limb = a.order ? a.order[t.limb0 + blockIdx.y] : t.limb0 + blockIdx.y;
    const uint32_t li = limb - t.limb0;
    const LimbDev lc = a.limbs[limb];
    const uint64_t S = ((uint64_t)t.n_ct * a.n_limbs) << (K1 + K2);   // elements per operand
    const uint64_t rowb = ((uint64_t)p * a.n_limbs + limb) << (K1 + K2);
    const uint32_t E = 1u << (K1 + K2 - logC);
    TileCtx col, row;
    cluster_ctx<false, K1, K2>(col, row, a, rank, nullptr, a.out + k * S + rowb, sm,
                               E >> LOG_R);

    const TensorK tk{lc.q, t.s[li], t.sp[li], lc.barrett_k, lc.barrett_qm1, t.in_mf};
    const uint64_t base = rowb + (row.b_base << K2);   // the CTA's rows are contiguous
    if (lc.narrow)
        cluster_tensor_tile<0, LOG_R>(sm, t, tk, base, S, k, row.nthreads);
    else if (lc.trunc)
        cluster_tensor_tile<1, LOG_R>(sm, t, tk, base, S, k, row.nthreads);
    else
        cluster_tensor_tile<2, LOG_R>(sm, t, tk, base, S, k, row.nthreads);
    __syncthreads();
    cluster_dispatch<false, LOG_R, K1, K2>(sm, lc, col, row);
}

typedef void (*ClusterKernel)(PassArgs);
typedef void (*ClusterTensorKernel)(PassArgs, TensorIn);

// ntt_cluster_f.cu / ntt_cluster_i.cu / ntt_cluster_t.cu: the menu of
// (elements per thread, column stages, row stages); nullptr if not built.
ClusterKernel pick_cluster_f(int logR, int K1, int K2);
ClusterKernel pick_cluster_i(int logR, int K1, int K2);
ClusterTensorKernel pick_cluster_t(int logR, int K1, int K2);

// The (K1, K2) pairs instantiated: N = 2^14 .. 2^17, both phases 6 .. 9 stages.
#define HX_CLUSTER_MENU(F)                                                           \
    F(6, 8) F(7, 7) F(8, 6) F(6, 9) F(7, 8) F(8, 7) F(9, 6) F(7, 9) F(8, 8) F(9, 7) \
    F(8, 9) F(9, 8)

}  // namespace hx
