// The element-wise ciphertext tensor fused into the first pass of the inverse
// transform (cross-kernel fusion of the multiply and FMA steps into the NTT,
// the direction Section 5 of the paper points to).
//
// The inverse's first pass is always a row pass that stages its input tile
// through shared memory.  Here that staging step computes the tile of
// r_k = (d_k s + e_k) mod q, d0 = A0 B0, d1 = A0 B1 + A1 B0, d2 = A1 B1,
// straight from the forward outputs A0, A1, B0, B1 and the addend e_k -- the
// values the element-wise tensor kernel computes, with fewer multiplies
// (tensor_r3 / tensor_rk: the scalar applied to a0 and a1 once, d1 by
// Karatsuba, 32-bit words for q < 2^30); the pass then runs its
// Gentleman-Sande rounds on it unchanged.  The three r_k never go to HBM,
// and the element-wise kernel's launch disappears.
#pragma once
#include "ntt_kernels.cuh"
#include "ntt_tensor.h"

namespace hx {

// The tile of r_k, two elements per step (16-byte loads; row passes cover
// whole rows, so the tile is contiguous from b_base << K), into shared memory
// for the rounds.  Wd: the limb's word class (tensor_r3).
template <int Wd, int LOG_R, int K, int NPF>
__device__ __forceinline__ void tensor_tile_to_smem(uint64_t* sm, const TensorIn& t,
                                                    const TensorK& tk, uint64_t base,
                                                    uint64_t S, uint32_t k, uint32_t nthreads,
                                                    uint32_t TEP) {
    const ulonglong2* A0 = reinterpret_cast<const ulonglong2*>(t.A + base);
    const ulonglong2* A1 = reinterpret_cast<const ulonglong2*>(t.A + S + base);
    const ulonglong2* B0 = reinterpret_cast<const ulonglong2*>(t.A + 2 * S + base);
    const ulonglong2* B1 = reinterpret_cast<const ulonglong2*>(t.A + 3 * S + base);
    const ulonglong2* E = reinterpret_cast<const ulonglong2*>(t.E + base);
    const ulonglong2 zero = make_ulonglong2(0, 0);
    // 2^(LOG_R-1) pairs a thread; a compile-time count lets the loads of
    // consecutive steps overlap (one step at a time for three outputs, whose
    // registers are already full)
#pragma unroll(NPF == 3 ? 1 : 4)
    for (int it = 0; it < (1 << (LOG_R - 1)); ++it) {
        const uint32_t i = threadIdx.x + it * nthreads;
        const uint32_t l = 2 * i;   // l even: l and l + 1 share one 16-word row
        if constexpr (NPF == 3) {
            const ulonglong2 x0 = __ldg(A0 + i), x1 = __ldg(A1 + i);
            const ulonglong2 y0 = __ldg(B0 + i), y1 = __ldg(B1 + i);
            const ulonglong2 e0 = __ldg(E + i), e1 = __ldg(E + S / 2 + i),
                             e2 = __ldg(E + S + i);
            tensor_r3<Wd>(x0.x, x1.x, y0.x, y1.x, e0.x, e1.x, e2.x, tk, sm[pad(l)],
                          sm[TEP + pad(l)], sm[2 * TEP + pad(l)]);
            tensor_r3<Wd>(x0.y, x1.y, y0.y, y1.y, e0.y, e1.y, e2.y, tk, sm[pad(l) + 1],
                          sm[TEP + pad(l) + 1], sm[2 * TEP + pad(l) + 1]);
        } else {
            const bool need0 = k != 2, need1 = k != 0;
            const ulonglong2 x0 = need0 ? __ldg(A0 + i) : zero;
            const ulonglong2 x1 = need1 ? __ldg(A1 + i) : zero;
            const ulonglong2 y0 = need0 ? __ldg(B0 + i) : zero;
            const ulonglong2 y1 = need1 ? __ldg(B1 + i) : zero;
            const ulonglong2 e = __ldg(E + k * (S / 2) + i);
            sm[pad(l)] = tensor_rk<Wd>(k, x0.x, x1.x, y0.x, y1.x, e.x, tk);
            sm[pad(l) + 1] = tensor_rk<Wd>(k, x0.y, x1.y, y0.y, y1.y, e.y, tk);
        }
    }
}

// The inverse stages on the block's output tiles in shared memory: one
// output, or three one after another (output kk's tile at sm + kk TEP, its
// HBM destination kk operands after the first).
template <typename Wd, int AR, int LOG_R, int K, int NPF, bool TWS>
__device__ __forceinline__ void tensor_rounds(uint64_t* sm, const ulonglong2* __restrict__ tw,
                                              const LimbDev& lc, const TileCtx& c, uint64_t S,
                                              uint32_t TEP) {
    if constexpr (NPF == 3) {
#pragma unroll 1
        for (int kk = 0; kk < 3; ++kk) {
            TileCtx ck = c;
            ck.gout = c.gout + kk * S;
            ck.np_valid = 1;
            ntt_rounds<false, false, Wd, AR, LOG_R, K, 0, 1, TWS>(sm + kk * TEP, tw, lc, ck);
        }
    } else {
        ntt_rounds<false, false, Wd, AR, LOG_R, K, 0, 1, TWS>(sm, tw, lc, c);
    }
}

// NPF = 1: one block per (tile, output k, ciphertext, limb); NPF = 3: one
// block per (tile, ciphertext, limb) computing all three r_k from one read of
// the operands, then transforming them one after another (the second and
// third output's twiddles come from L1).
// Register caps (measured on GB300 at N = 2^16 x 32 limbs): HX_TENSOR3_MAXNREG
// for three outputs a block, and as the per-tile passes for one output a
// block.  Transforming the three outputs together (every twiddle load serving
// three butterflies) needed 96 registers, five blocks of 128 threads per SM;
// one output at a time fits 72, seven blocks: the tensor + inverse call
// 96.4 -> 90.3 us (64: 94.3 us, 56: 96.2 us).  Blocks have at most 512
// threads.
#ifndef HX_TENSOR3_MAXNREG
#define HX_TENSOR3_MAXNREG 72
#endif
template <int LOG_R, int K, bool TWS, int NPF>
__global__ void __maxnreg__(NPF == 3 ? HX_TENSOR3_MAXNREG : (LOG_R == 4 ? 72 : 64))
    ntt_tensor_inv_kernel(PassArgs a, TensorIn t) {
    extern __shared__ uint64_t sm[];
    const uint32_t limb = a.order ? a.order[t.limb0 + blockIdx.y] : t.limb0 + blockIdx.y;
    const uint32_t li = limb - t.limb0;
    const uint32_t G = (NPF == 3 ? 1 : 3) * t.n_ct;
    const uint32_t g = blockIdx.x % G, tile = blockIdx.x / G;
    const uint32_t k = NPF == 3 ? 0 : g / t.n_ct, p = g % t.n_ct;
    const LimbDev lc = a.limbs[limb];
    const uint64_t S = ((uint64_t)t.n_ct * a.n_limbs) << a.L;   // elements per operand
    const uint64_t row = ((uint64_t)p * a.n_limbs + limb) << a.L;
    const uint32_t TE = 1u << (a.logGb + K);
    TileCtx c;
    c.gin = nullptr;
    c.gout = a.out + k * S + row;
    c.b_base = (uint64_t)tile << a.logGb;
    c.c_base = 0;
    c.L = a.L;
    c.s0 = a.s0;
    c.logGc = 0;
    c.logGb = a.logGb;
    c.w = 0;
    c.nthreads = TE >> LOG_R;
    c.out_mf = a.out_mf;
    c.last = a.last != 0;
    c.poly_stride = S;
    c.np_valid = NPF;

    const ulonglong2* tw = lc.inv;
    if constexpr (TWS) {
        ulonglong2* tws = reinterpret_cast<ulonglong2*>(sm + NPF * padded(TE));
        stage_twiddles<K, LOG_R>(tws, tw, c);
        cp_async_commit();
        tw = tws;
    }

    const TensorK tk{lc.q, t.s[li], t.sp[li], lc.barrett_k, lc.barrett_qm1, t.in_mf};
    const uint64_t base = row + (c.b_base << K);
    const uint32_t TEP = padded(TE);
    if (lc.narrow) {
        tensor_tile_to_smem<0, LOG_R, K, NPF>(sm, t, tk, base, S, k, c.nthreads, TEP);
        if constexpr (TWS) cp_async_wait<0>();
        __syncthreads();
        tensor_rounds<uint32_t, 0, LOG_R, K, NPF, TWS>(sm, tw, lc, c, S, TEP);
    } else if (lc.trunc) {
        tensor_tile_to_smem<1, LOG_R, K, NPF>(sm, t, tk, base, S, k, c.nthreads, TEP);
        if constexpr (TWS) cp_async_wait<0>();
        __syncthreads();
        tensor_rounds<uint64_t, 1, LOG_R, K, NPF, TWS>(sm, tw, lc, c, S, TEP);
    } else {
        tensor_tile_to_smem<2, LOG_R, K, NPF>(sm, t, tk, base, S, k, c.nthreads, TEP);
        if constexpr (TWS) cp_async_wait<0>();
        __syncthreads();
        tensor_rounds<uint64_t, 0, LOG_R, K, NPF, TWS>(sm, tw, lc, c, S, TEP);
    }
}

template <int LOG_R, bool TWS, int NPF>
inline TensorPassKernel tensor_k(int K) {
    switch (K) {
        case 6: return ntt_tensor_inv_kernel<LOG_R, 6, TWS, NPF>;
        case 7: return ntt_tensor_inv_kernel<LOG_R, 7, TWS, NPF>;
        case 8: return ntt_tensor_inv_kernel<LOG_R, 8, TWS, NPF>;
        case 9: return ntt_tensor_inv_kernel<LOG_R, 9, TWS, NPF>;
        case 10: return ntt_tensor_inv_kernel<LOG_R, 10, TWS, NPF>;
        case 11: return ntt_tensor_inv_kernel<LOG_R, 11, TWS, NPF>;
        case 12: return ntt_tensor_inv_kernel<LOG_R, 12, TWS, NPF>;
        case 13: return ntt_tensor_inv_kernel<LOG_R, 13, TWS, NPF>;
        default: return nullptr;
    }
}

}  // namespace hx
