// The ciphertext tensor step with the forward's and the inverse's row passes
// fused around it (cross-kernel fusion, the direction Section 5 of the paper
// points to, one step beyond ntt_tensor.cuh): one block per (row tile,
// ciphertext, limb) runs the forward's row stages on its tiles of A0, A1, B0
// and B1 -- read from the forward's column pass output -- one spectrum after
// another, keeps the four spectra in shared memory, computes
// r_k = (d_k s + e_k) mod q there (tensor_r3), and runs the inverse's row
// stages on the three r_k one after another, writing them for the inverse's
// column pass.  The four spectra never go to HBM: the forward's row pass does
// not write them and the fused pass does not read them back.
#include <type_traits>

#include "ntt_tensor.cuh"

namespace hx {

#ifndef HX_CTROW_MAXNREG
#define HX_CTROW_MAXNREG 72
#endif

// WC: the limb's word class (tensor_r3): 0 32-bit words, 1 64-bit words with
// truncated quotients, 2 64-bit words with exact ones.
template <int WC, int LOG_R, int K>
__device__ __forceinline__ void ct_row_body(uint64_t* sm, const LimbDev& lc, TileCtx cf,
                                            const TileCtx& ci, const TensorIn& t,
                                            const TensorK& tk, uint64_t base, uint64_t S,
                                            uint32_t TEP) {
    using Wd = typename std::conditional<WC == 0, uint32_t, uint64_t>::type;
    constexpr int AR = WC == 1 ? 1 : 0;
    // forward stages s0 .. L-1 of each spectrum: the first round reads the
    // tile from HBM, the last leaves it (below 4q) in its shared tile
#pragma unroll 1
    for (int o = 0; o < 4; ++o) {
        ntt_rounds<true, false, Wd, AR, LOG_R, K, 0, 1, false>(sm + o * TEP, lc.fwd, lc, cf);
        cf.gin += S;
    }
    __syncthreads();
    // the tensor step on the spectra, in place: position l of r_k replaces
    // position l of the k-th tile (each position is one thread's)
    const ulonglong2* E = reinterpret_cast<const ulonglong2*>(t.E + base);
#pragma unroll 1
    for (int it = 0; it < (1 << (LOG_R - 1)); ++it) {
        const uint32_t i = threadIdx.x + it * cf.nthreads;
        const uint32_t l = pad(2 * i);   // 2i even: 2i and 2i + 1 share one 16-word row
        const ulonglong2 e0 = __ldg(E + i), e1 = __ldg(E + S / 2 + i), e2 = __ldg(E + S + i);
        const uint64_t a0x = sm[l], a0y = sm[l + 1];
        const uint64_t a1x = sm[TEP + l], a1y = sm[TEP + l + 1];
        const uint64_t b0x = sm[2 * TEP + l], b0y = sm[2 * TEP + l + 1];
        const uint64_t b1x = sm[3 * TEP + l], b1y = sm[3 * TEP + l + 1];
        tensor_r3<WC>(a0x, a1x, b0x, b1x, e0.x, e1.x, e2.x, tk, sm[l], sm[TEP + l],
                      sm[2 * TEP + l]);
        tensor_r3<WC>(a0y, a1y, b0y, b1y, e0.y, e1.y, e2.y, tk, sm[l + 1], sm[TEP + l + 1],
                      sm[2 * TEP + l + 1]);
    }
    __syncthreads();
    // inverse stages L-1 .. s0 of r_0, r_1, r_2, one after another
    tensor_rounds<Wd, AR, LOG_R, K, 3, false>(sm, lc.inv, lc, ci, S, TEP);
}

// Grid (tiles x n_ct, limbs of the launch), 2^(logGb+K-LOG_R) threads,
// 4 padded tiles of shared memory.  t.A: the forward column pass's output
// of A0 | A1 | B0 | B1 back to back; t.E the addends; a.out the r_k after
// the inverse's row stages; a.s0 = L - K (the row passes' first stage).
template <int LOG_R, int K>
__global__ void __maxnreg__(HX_CTROW_MAXNREG) ntt_ct_row_kernel(PassArgs a, TensorIn t) {
    extern __shared__ uint64_t sm[];
    const uint32_t limb = a.order ? a.order[t.limb0 + blockIdx.y] : t.limb0 + blockIdx.y;
    const uint32_t li = limb - t.limb0;
    const uint32_t p = blockIdx.x % t.n_ct, tile = blockIdx.x / t.n_ct;
    const LimbDev lc = a.limbs[limb];
    const uint64_t S = ((uint64_t)t.n_ct * a.n_limbs) << a.L;   // elements per operand
    const uint64_t row = ((uint64_t)p * a.n_limbs + limb) << a.L;
    const uint32_t TE = 1u << (a.logGb + K);
    TileCtx cf;
    cf.gin = t.A + row;
    cf.gout = nullptr;
    cf.b_base = (uint64_t)tile << a.logGb;
    cf.c_base = 0;
    cf.L = a.L;
    cf.s0 = a.s0;
    cf.logGc = 0;
    cf.logGb = a.logGb;
    cf.w = 0;
    cf.nthreads = TE >> LOG_R;
    cf.out_mf = 4;      // the forward's outputs, as the tensor step takes them
    cf.last = true;
    cf.poly_stride = S;
    cf.np_valid = 1;
    TileCtx ci = cf;
    ci.gin = nullptr;
    ci.gout = a.out + row;
    ci.out_mf = a.out_mf;
    ci.last = a.last != 0;
    const TensorK tk{lc.q, t.s[li], t.sp[li], lc.barrett_k, lc.barrett_qm1, 4};
    const uint64_t base = row + (cf.b_base << K);
    const uint32_t TEP = padded(TE);
    if (lc.narrow)
        ct_row_body<0, LOG_R, K>(sm, lc, cf, ci, t, tk, base, S, TEP);
    else if (lc.trunc)
        ct_row_body<1, LOG_R, K>(sm, lc, cf, ci, t, tk, base, S, TEP);
    else
        ct_row_body<2, LOG_R, K>(sm, lc, cf, ci, t, tk, base, S, TEP);
}

// The polynomial product (Listing 4) the same way: one block per (row tile,
// polynomial, limb) runs the forward's row stages on its tiles of a and b
// (from the forward column pass's output, a.in = a | b back to back), forms
// c_i = a_i b_i mod q in shared memory (mulmod_fused, the value
// EltwiseMultMod gives) and runs the inverse's row stages on c, writing it for
// the inverse's column pass.  Neither spectrum nor the product reaches HBM.
#ifndef HX_MULROW_MAXNREG
#define HX_MULROW_MAXNREG 64
#endif

template <int WC, int LOG_R, int K>
__device__ __forceinline__ void mul_row_body(uint64_t* sm, const LimbDev& lc, TileCtx cf,
                                             const TileCtx& ci, uint64_t S, uint32_t TEP) {
    using Wd = typename std::conditional<WC == 0, uint32_t, uint64_t>::type;
    constexpr int AR = WC == 1 ? 1 : 0;
#pragma unroll 1
    for (int o = 0; o < 2; ++o) {
        ntt_rounds<true, false, Wd, AR, LOG_R, K, 0, 1, false>(sm + o * TEP, lc.fwd, lc, cf);
        cf.gin += S;
    }
    __syncthreads();
    const uint64_t q = lc.q, bk = lc.barrett_k;
    const uint32_t Qm1 = lc.barrett_qm1;
#pragma unroll 1
    for (int it = 0; it < (1 << (LOG_R - 1)); ++it) {
        const uint32_t l = pad(2 * (threadIdx.x + it * cf.nthreads));
#pragma unroll
        for (int h = 0; h < 2; ++h)   // the spectra are below 4q (the forward's out range)
            sm[l + h] = mulmod_fused<WC>(small_mod_rt(sm[l + h], q, 4),
                                         small_mod_rt(sm[TEP + l + h], q, 4), q, bk, Qm1);
    }
    __syncthreads();
    ntt_rounds<false, false, Wd, AR, LOG_R, K, 0, 1, false>(sm, lc.inv, lc, ci);
}

// Grid (tiles x n_polys, limbs), 2^(logGb+K-LOG_R) threads, two padded tiles
// of shared memory; a.n_polys products, a.s0 = L - K.
template <int LOG_R, int K>
__global__ void __maxnreg__(HX_MULROW_MAXNREG) ntt_mul_row_kernel(PassArgs a) {
    extern __shared__ uint64_t sm[];
    const uint32_t limb = a.order ? a.order[blockIdx.y] : blockIdx.y;
    const uint32_t p = blockIdx.x % a.n_polys, tile = blockIdx.x / a.n_polys;
    const LimbDev lc = a.limbs[limb];
    const uint64_t S = ((uint64_t)a.n_polys * a.n_limbs) << a.L;   // elements per operand
    const uint64_t row = ((uint64_t)p * a.n_limbs + limb) << a.L;
    const uint32_t TE = 1u << (a.logGb + K);
    TileCtx cf;
    cf.gin = a.in + row;
    cf.gout = nullptr;
    cf.b_base = (uint64_t)tile << a.logGb;
    cf.c_base = 0;
    cf.L = a.L;
    cf.s0 = a.s0;
    cf.logGc = 0;
    cf.logGb = a.logGb;
    cf.w = 0;
    cf.nthreads = TE >> LOG_R;
    cf.out_mf = 4;
    cf.last = true;
    cf.poly_stride = S;
    cf.np_valid = 1;
    TileCtx ci = cf;
    ci.gin = nullptr;
    ci.gout = a.out + row;
    ci.out_mf = a.out_mf;
    ci.last = a.last != 0;
    const uint32_t TEP = padded(TE);
    if (lc.narrow)
        mul_row_body<0, LOG_R, K>(sm, lc, cf, ci, S, TEP);
    else if (lc.trunc)
        mul_row_body<1, LOG_R, K>(sm, lc, cf, ci, S, TEP);
    else
        mul_row_body<2, LOG_R, K>(sm, lc, cf, ci, S, TEP);
}

PassKernel pick_mul_row(int logR, int K) {
    if (logR != 3) return nullptr;
    switch (K) {
        case 6: return ntt_mul_row_kernel<3, 6>;
        case 7: return ntt_mul_row_kernel<3, 7>;
        case 8: return ntt_mul_row_kernel<3, 8>;
        case 9: return ntt_mul_row_kernel<3, 9>;
        default: return nullptr;
    }
}

TensorPassKernel pick_ct_row(int logR, int K) {
    if (logR != 3) return nullptr;
    switch (K) {
        case 6: return ntt_ct_row_kernel<3, 6>;
        case 7: return ntt_ct_row_kernel<3, 7>;
        case 8: return ntt_ct_row_kernel<3, 8>;
        case 9: return ntt_ct_row_kernel<3, 9>;
        default: return nullptr;
    }
}

}  // namespace hx
