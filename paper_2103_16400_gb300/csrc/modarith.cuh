// Device modular arithmetic for word-sized primes (Sections 2.1-2.2 and 3.2
// of Intel HEXL, arXiv 2103.16400), written for the 32-bit integer multiply
// pipes of sm_103a.
//
// Two widths, chosen per modulus (the paper's BitShift idea, Section 3.2):
//   * wide  : q < 2^62, words of beta = 2^64; a Shoup product needs the high
//             word of a 64x64 product plus two low words.
//   * narrow: q < 2^30, words of beta = 2^32; the Shoup product is three 32-bit
//             multiplies (one high half, two low halves).
// The Harvey butterflies (Section 2.2) need q < beta/4 in both cases.
#pragma once
#include <stdint.h>

namespace hx {

// ---------------------------------------------------------------- 64-bit words
__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
    return __umul64hi(a, b);
}

// Shoup modular product (Algorithms "Harvey NTT butterfly" and
// "Harvey inverse NTT butterfly"): with wp = floor(w * 2^64 / q) and any
// x < 2^64, returns w*x mod q up to one extra q, i.e. a value in [0, 2q).
__device__ __forceinline__ uint64_t shoup_mul_lazy64(uint64_t x, uint64_t w, uint64_t wp,
                                                     uint64_t q) {
    uint64_t Q = mulhi64(wp, x);
    return w * x - Q * q;
}

// Harvey forward butterfly: X0, X1 in [0, 4q) -> X0 + W X1, X0 - W X1 in [0, 4q).
__device__ __forceinline__ void harvey_fwd64(uint64_t& X0, uint64_t& X1, uint64_t W,
                                             uint64_t Wp, uint64_t q, uint64_t two_q) {
    uint64_t x0 = X0 >= two_q ? X0 - two_q : X0;
    uint64_t T = shoup_mul_lazy64(X1, W, Wp, q);
    X0 = x0 + T;
    X1 = x0 - T + two_q;
}

// Harvey inverse butterfly: X0, X1 in [0, 2q) -> X0 + X1, W (X0 - X1) in [0, 2q).
__device__ __forceinline__ void harvey_inv64(uint64_t& X0, uint64_t& X1, uint64_t W,
                                             uint64_t Wp, uint64_t q, uint64_t two_q) {
    uint64_t y0 = X0 + X1;
    y0 = y0 >= two_q ? y0 - two_q : y0;
    uint64_t T = X0 - X1 + two_q;
    X1 = shoup_mul_lazy64(T, W, Wp, q);
    X0 = y0;
}

// ---------------------------------------------------------------- 32-bit words
__device__ __forceinline__ uint32_t shoup_mul_lazy32(uint32_t x, uint32_t w, uint32_t wp,
                                                     uint32_t q) {
    uint32_t Q = __umulhi(wp, x);
    return w * x - Q * q;
}

__device__ __forceinline__ void harvey_fwd32(uint32_t& X0, uint32_t& X1, uint32_t W,
                                             uint32_t Wp, uint32_t q, uint32_t two_q) {
    uint32_t x0 = X0 >= two_q ? X0 - two_q : X0;
    uint32_t T = shoup_mul_lazy32(X1, W, Wp, q);
    X0 = x0 + T;
    X1 = x0 - T + two_q;
}

__device__ __forceinline__ void harvey_inv32(uint32_t& X0, uint32_t& X1, uint32_t W,
                                             uint32_t Wp, uint32_t q, uint32_t two_q) {
    uint32_t y0 = X0 + X1;
    y0 = y0 >= two_q ? y0 - two_q : y0;
    uint32_t T = X0 - X1 + two_q;
    X1 = shoup_mul_lazy32(T, W, Wp, q);
    X0 = y0;
}

// ---------------------------------------------------------------- reductions
// x in [0, k q) -> x mod q for k in {1, 2, 4, 8}, by log2(k) conditional
// subtractions of 4q, 2q, q (the paper's small_mod, Section 3.2).
template <int K>
__device__ __forceinline__ uint64_t small_mod(uint64_t x, uint64_t q) {
    if (K >= 8) x = x >= 4 * q ? x - 4 * q : x;
    if (K >= 4) x = x >= 2 * q ? x - 2 * q : x;
    if (K >= 2) x = x >= q ? x - q : x;
    return x;
}

__device__ __forceinline__ uint64_t small_mod_rt(uint64_t x, uint64_t q, uint32_t k) {
    if (k >= 8) x = x >= 4 * q ? x - 4 * q : x;
    if (k >= 4) x = x >= 2 * q ? x - 2 * q : x;
    if (k >= 2) x = x >= q ? x - q : x;
    return x;
}

// Barrett reduction of a 128-bit d = (hi, lo) < 2^(2Q+1) (Algorithm "Barrett
// Reduction" with Q = bitlen(q), L = 63 + Q, k = floor(2^L / q), so that
// c3 is the high word of c1 * k).  The quotient estimate c3 is short of
// floor(d / q) by at most 2, so two conditional subtractions finish it.
struct Barrett {
    uint64_t q;
    uint64_t k;      // floor(2^(63+Q) / q)
    uint32_t Qm1;    // Q - 1, the right shift that forms c1
};

__device__ __forceinline__ uint64_t barrett_reduce128(uint64_t hi, uint64_t lo,
                                                      const Barrett& b) {
    // c1 = d >> (Q - 1); Q - 1 is in [1, 61]
    uint64_t c1 = (lo >> b.Qm1) | (hi << (64 - b.Qm1));
    uint64_t c3 = mulhi64(c1, b.k);
    uint64_t c4 = lo - c3 * b.q;
    c4 = c4 >= b.q ? c4 - b.q : c4;
    c4 = c4 >= b.q ? c4 - b.q : c4;
    return c4;
}

__device__ __forceinline__ uint64_t barrett_mulmod(uint64_t x, uint64_t y, const Barrett& b) {
    return barrett_reduce128(mulhi64(x, y), x * y, b);
}

}  // namespace hx
