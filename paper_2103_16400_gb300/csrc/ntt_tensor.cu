// The element-wise ciphertext tensor fused into the first pass of the inverse
// transform (cross-kernel fusion of the multiply and FMA steps into the NTT,
// the direction Section 5 of the paper points to).
//
// The inverse's first pass is always a row pass that stages its input tile
// through shared memory.  Here that staging step computes the tile of
// r_k = (d_k s + e_k) mod q, d0 = A0 B0, d1 = A0 B1 + A1 B0, d2 = A1 B1,
// straight from the forward outputs A0, A1, B0, B1 and the addend e_k, with
// the same arithmetic as the element-wise tensor kernel (tensor_d, tensor_r);
// the pass then runs its Gentleman-Sande rounds on it unchanged.  The three
// r_k never go to HBM, and the element-wise kernel's launch disappears.
#include "ntt_kernels.cuh"
#include "ntt_tensor.h"

namespace hx {

template <int LOG_R, int K, bool TWS>
__global__ void __launch_bounds__(512) ntt_tensor_inv_kernel(PassArgs a, TensorIn t) {
    extern __shared__ uint64_t sm[];
    const uint32_t li = blockIdx.y, limb = t.limb0 + li;
    const uint32_t G = 3 * t.n_ct;
    const uint32_t g = blockIdx.x % G, tile = blockIdx.x / G;
    const uint32_t k = g / t.n_ct, p = g % t.n_ct;
    const LimbDev lc = a.limbs[limb];
    const uint64_t S = ((uint64_t)t.n_ct * a.n_limbs) << a.L;   // elements per operand
    const uint64_t row = ((uint64_t)p * a.n_limbs + limb) << a.L;
    const uint32_t TE = 1u << (a.logGb + K);
    TileCtx c;
    c.gin = nullptr;
    c.gout = a.out + (((uint64_t)g * a.n_limbs + limb) << a.L);
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

    const ulonglong2* tw = lc.inv;
    if constexpr (TWS) {
        ulonglong2* tws = reinterpret_cast<ulonglong2*>(sm + padded(TE));
        stage_twiddles<K, LOG_R>(tws, tw, c);
        cp_async_commit();
        tw = tws;
    }

    // the tile of r_k, two elements per step (16-byte loads; row passes
    // cover whole rows, so the tile is contiguous from b_base << K)
    const uint64_t q = lc.q;
    const Barrett br{q, lc.barrett_k, lc.barrett_qm1};
    const uint64_t s = t.s[li], sp = t.sp[li];
    const uint64_t base = row + (c.b_base << K);
    const ulonglong2* A0 = reinterpret_cast<const ulonglong2*>(t.A + base);
    const ulonglong2* A1 = reinterpret_cast<const ulonglong2*>(t.A + S + base);
    const ulonglong2* B0 = reinterpret_cast<const ulonglong2*>(t.A + 2 * S + base);
    const ulonglong2* B1 = reinterpret_cast<const ulonglong2*>(t.A + 3 * S + base);
    const ulonglong2* Ek = reinterpret_cast<const ulonglong2*>(t.E + k * S + base);
    const ulonglong2 zero = make_ulonglong2(0, 0);
    for (uint32_t i = threadIdx.x; i < TE / 2; i += c.nthreads) {
        const ulonglong2 x0 = k != 2 ? __ldg(A0 + i) : zero;
        const ulonglong2 x1 = k != 0 ? __ldg(A1 + i) : zero;
        const ulonglong2 y0 = k != 2 ? __ldg(B0 + i) : zero;
        const ulonglong2 y1 = k != 0 ? __ldg(B1 + i) : zero;
        const ulonglong2 e = __ldg(Ek + i);
        const uint64_t r0 = tensor_r(tensor_d(k, small_mod_rt(x0.x, q, t.in_mf),
                                              small_mod_rt(x1.x, q, t.in_mf),
                                              small_mod_rt(y0.x, q, t.in_mf),
                                              small_mod_rt(y1.x, q, t.in_mf), br),
                                     e.x, s, sp, q);
        const uint64_t r1 = tensor_r(tensor_d(k, small_mod_rt(x0.y, q, t.in_mf),
                                              small_mod_rt(x1.y, q, t.in_mf),
                                              small_mod_rt(y0.y, q, t.in_mf),
                                              small_mod_rt(y1.y, q, t.in_mf), br),
                                     e.y, s, sp, q);
        const uint32_t l = 2 * i;
        sm[pad(l)] = r0;   // l even: l and l + 1 share one 16-word row
        sm[pad(l) + 1] = r1;
    }
    if constexpr (TWS) cp_async_wait<0>();
    __syncthreads();
    if (lc.narrow)
        ntt_rounds<false, false, uint32_t, 0, LOG_R, K, 0, 1, TWS>(sm, tw, lc, c);
    else if (lc.trunc)
        ntt_rounds<false, false, uint64_t, 1, LOG_R, K, 0, 1, TWS>(sm, tw, lc, c);
    else
        ntt_rounds<false, false, uint64_t, 0, LOG_R, K, 0, 1, TWS>(sm, tw, lc, c);
}

template <int LOG_R, bool TWS>
static TensorPassKernel tensor_k(int K) {
    switch (K) {
        case 6: return ntt_tensor_inv_kernel<LOG_R, 6, TWS>;
        case 7: return ntt_tensor_inv_kernel<LOG_R, 7, TWS>;
        case 8: return ntt_tensor_inv_kernel<LOG_R, 8, TWS>;
        case 9: return ntt_tensor_inv_kernel<LOG_R, 9, TWS>;
        case 10: return ntt_tensor_inv_kernel<LOG_R, 10, TWS>;
        case 11: return ntt_tensor_inv_kernel<LOG_R, 11, TWS>;
        case 12: return ntt_tensor_inv_kernel<LOG_R, 12, TWS>;
        case 13: return ntt_tensor_inv_kernel<LOG_R, 13, TWS>;
        default: return nullptr;
    }
}

TensorPassKernel pick_tensor_inv(int logR, int K, bool tws) {
    if (logR == 3) return tws ? tensor_k<3, true>(K) : tensor_k<3, false>(K);
    if (logR == 4) return tws ? tensor_k<4, true>(K) : tensor_k<4, false>(K);
    return nullptr;
}

}  // namespace hx
