// Device modular arithmetic for word-sized primes (Sections 2.1-2.2 and 3.2
// of Intel HEXL, arXiv 2103.16400), written for the 32-bit integer multiply
// pipes of sm_103a.
//
// Two widths, chosen per modulus (the paper's BitShift idea, Section 3.2):
//   * wide  : q < 2^62, words of beta = 2^64; a Shoup product needs the high
//             word of a 64x64 product plus two low words.  Below 2^61 the high
//             word is truncated to three partial products (lazy bound 4q).
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

// The same product built explicitly from 32-bit multiplies, keeping carries
// and the final subtraction on the integer-multiply pipe rather than the ALU:
//
//   high word of a*b, a = a1:a0, b = b1:b0 (32-bit halves):
//     u = a0 b1 + hi(a0 b0)         < 2^64, no carry out
//     v = a1 b0 + lo32(u)           < 2^64
//     r = a1 b1 + hi32(u) + hi32(v)
//   (mul.hi + three mad.wide + one 64-bit add), or as a mad.lo.cc/madc.hi
//   carry chain over the same four partial products;
//
//   T = W X - Q q mod 2^64 = W X + Q (2^64 - q) mod 2^64: only the low word is
//   needed, so T = w0 x0 + Q0 n0 (two wide products summed mod 2^64) plus
//   2^32 (w0 x1 + w1 x0 + Q0 n1 + Q1 n0) mod 2^64 (four low-half mads).
__device__ __forceinline__ uint64_t mulhi64_wide(uint64_t a, uint64_t b) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint32_t h;
    uint64_t u, v, r;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(h) : "r"(a0), "r"(b0));
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(u) : "r"(a0), "r"(b1), "l"((uint64_t)h));
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(v) : "r"(a1), "r"(b0), "l"(u & 0xffffffffull));
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a1), "r"(b1), "l"(u >> 32));
    return r + (v >> 32);
}

__device__ __forceinline__ uint64_t mulhi64_cc(uint64_t a, uint64_t b) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint32_t r0, r1;
    asm("{\n\t.reg .u32 h, m;\n\t"
        "mul.hi.u32 h, %2, %4;\n\t"
        "mad.lo.cc.u32 h, %2, %5, h;\n\t"
        "madc.hi.u32 m, %2, %5, 0;\n\t"
        "mad.lo.cc.u32 h, %3, %4, h;\n\t"
        "madc.hi.cc.u32 m, %3, %4, m;\n\t"
        "madc.hi.u32 %1, %3, %5, 0;\n\t"
        "mad.lo.cc.u32 %0, %3, %5, m;\n\t"
        "addc.u32 %1, %1, 0;\n\t}"
        : "=r"(r0), "=r"(r1)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    return ((uint64_t)r1 << 32) | r0;
}

// (w x + Q nq) mod 2^64 with nq = 2^64 - q: the Shoup remainder W X - Q q.
__device__ __forceinline__ uint64_t shoup_rem64(uint64_t w, uint64_t x, uint64_t Q,
                                                uint64_t nq) {
    const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32);
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    const uint32_t Q0 = (uint32_t)Q, Q1 = (uint32_t)(Q >> 32);
    const uint32_t n0 = (uint32_t)nq, n1 = (uint32_t)(nq >> 32);
    uint64_t t;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(t) : "r"(w0), "r"(x0));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(t) : "r"(Q0), "r"(n0));
    uint32_t th = (uint32_t)(t >> 32);
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(th) : "r"(w0), "r"(x1));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(th) : "r"(w1), "r"(x0));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(th) : "r"(Q0), "r"(n1));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(th) : "r"(Q1), "r"(n0));
    return ((uint64_t)th << 32) | (uint32_t)t;
}

// Truncated high word of a*b: a1 b1 + hi32(a1 b0) + hi32(a0 b1), from three of
// the four partial products and no carry propagation out of the low word.
// The dropped part, (lo32(a1 b0) + lo32(a0 b1)) 2^32 + a0 b0, is below
// 3 * 2^64, so the result is floor(a b / 2^64) minus 0, 1 or 2.
__device__ __forceinline__ uint64_t mulhi64_trunc(uint64_t a, uint64_t b) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint32_t h0, h1;
    uint64_t r;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(h0) : "r"(a1), "r"(b0));
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(h1) : "r"(a0), "r"(b1));
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a1), "r"(b1), "l"((uint64_t)h0));
    return r + h1;
}

// Shoup product variants (V): 0 plain C++; 1 mad.wide high word + explicit
// remainder; 2 carry-chain high word + explicit remainder -- all three return
// the same value, w x mod q in [0, 2q); 3 truncated high word + explicit
// remainder.  With Q' = Q - e (e <= 2) the remainder W X - Q' q is the exact
// one plus e q, so variant 3 returns w x mod q in [0, 4q) (needs 4q < 2^64).
template <int V>
__device__ __forceinline__ uint64_t shoup_lazy64v(uint64_t x, uint64_t w, uint64_t wp, uint64_t q,
                                                  uint64_t nq) {
    if constexpr (V == 0) {
        return shoup_mul_lazy64(x, w, wp, q);
    } else {
        const uint64_t Q = V == 1 ? mulhi64_wide(wp, x)
                                  : V == 2 ? mulhi64_cc(wp, x) : mulhi64_trunc(wp, x);
        return shoup_rem64(w, x, Q, nq);
    }
}

#ifndef HX_SHOUP_VARIANT
#define HX_SHOUP_VARIANT 2
#endif

// x in [0, 2m) -> [0, m) (m = 2q or 4q): subtract m unless that borrows.
// Since m <= 2^63 and x < 2m, x - m wraps past 2^63 exactly when x < m, so
// the sign bit of the difference decides.
__device__ __forceinline__ uint64_t reduce_2q(uint64_t x, uint64_t two_q) {
    const uint64_t d = x - two_q;
    return (int64_t)d < 0 ? x : d;
}

// Harvey forward butterfly with lazy bound m, the range of the Shoup product
// (m = 2q for variants 0-2, m = 4q for variant 3):
// X0, X1 in [0, 2m) -> X0 + W X1, X0 - W X1 in [0, 2m).  Needs 2m < 2^64.
template <int V = HX_SHOUP_VARIANT>
__device__ __forceinline__ void harvey_fwd64(uint64_t& X0, uint64_t& X1, uint64_t W,
                                             uint64_t Wp, uint64_t q, uint64_t m) {
    const uint64_t x0 = V == 0 ? (X0 >= m ? X0 - m : X0) : reduce_2q(X0, m);
    const uint64_t T = shoup_lazy64v<V>(X1, W, Wp, q, 0 - q);
    X0 = x0 + T;
    X1 = x0 - T + m;
}

// Harvey inverse butterfly with lazy bound m (as above):
// X0, X1 in [0, m) -> X0 + X1, W (X0 - X1) in [0, m).
template <int V = HX_SHOUP_VARIANT>
__device__ __forceinline__ void harvey_inv64(uint64_t& X0, uint64_t& X1, uint64_t W,
                                             uint64_t Wp, uint64_t q, uint64_t m) {
    uint64_t y0 = X0 + X1;
    y0 = V == 0 ? (y0 >= m ? y0 - m : y0) : reduce_2q(y0, m);
    const uint64_t T = X0 - X1 + m;
    X1 = shoup_lazy64v<V>(T, W, Wp, q, 0 - q);
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

// a s mod q in [0, q) for a < 2^64, s < q, sp = floor(s 2^64 / q): the Shoup
// product of Algorithm "EltwiseFMAModAVX512" ([0, 2q)) and one subtraction.
__device__ __forceinline__ uint64_t fma_shoup(uint64_t a, uint64_t s, uint64_t sp, uint64_t q) {
    uint64_t r = s * a - mulhi64(sp, a) * q;  // [0, 2q)
    return r >= q ? r - q : r;
}

// ---------------------------------------------------------------- ciphertext tensor
// Term k of the element-wise ciphertext tensor from residues in [0, q):
// d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 (mod q).  d1 reduces the
// 128-bit sum of the two products (< 2 q^2 < 2^(2Q+1)) with one Barrett.
__device__ __forceinline__ uint64_t tensor_d(uint32_t k, uint64_t a0, uint64_t a1, uint64_t b0,
                                             uint64_t b1, const Barrett& br) {
    if (k == 0) return barrett_mulmod(a0, b0, br);
    if (k == 2) return barrett_mulmod(a1, b1, br);
    uint64_t lo = a0 * b1, hi = mulhi64(a0, b1);
    const uint64_t lo2 = a1 * b0, hi2 = mulhi64(a1, b0);
    lo += lo2;
    hi += hi2 + (lo < lo2 ? 1 : 0);
    return barrett_reduce128(hi, lo, br);
}

// r = d s + e mod q in [0, q) (EltwiseFMAMod with addend), d, e in [0, q).
__device__ __forceinline__ uint64_t tensor_r(uint64_t d, uint64_t e, uint64_t s, uint64_t sp,
                                             uint64_t q) {
    const uint64_t t = fma_shoup(d, s, sp, q) + e;
    return t >= q ? t - q : t;
}


// ---------------------------------------------------------------- ciphertext tensor, fused form
// The fused inverse passes compute the same r_k = (d_k s + e_k) mod q with
// fewer multiplies.  The scalar is applied once to each of a0 and a1
// (a' = a s mod q, a Shoup product: s is fixed per limb), so that
//   r0 = a0' b0 + e0,  r2 = a1' b1 + e2,  r1 = a0' b1 + a1' b0 + e1   (mod q)
// take one Barrett reduction each and no FMA, and d1's two products come
// from one more: (a0' + a1')(b0 + b1) - a0' b0 - a1' b1, exact in 128 bits
// (Karatsuba).  Every r_k is returned in [0, q), the value the element-wise
// tensor (tensor_d, tensor_r) returns.
struct TensorK {
    uint64_t q, s, sp;   // modulus, scalar s < q, floor(s 2^64 / q)
    uint64_t bk;         // Barrett factor floor(2^(63+Q) / q), Q = bitlen(q)
    uint32_t Qm1;        // Q - 1
    uint32_t mf;         // input_mod_factor of the operands: 1, 2 or 4
};

// The 128-bit product a b from four 32x32-bit products (mad.wide):
// a b = p + 2^32 (a0 b1 + a1 b0) + 2^64 a1 b1 with p = a0 b0; the partial
// sums u = a0 b1 + hi32(p) and v = a1 b0 + lo32(u) stay below 2^64.
__device__ __forceinline__ void mul_full64(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint64_t p, u, v, r;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a0), "r"(b0));
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(u) : "r"(a0), "r"(b1), "l"(p >> 32));
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(v) : "r"(a1), "r"(b0), "l"(u & 0xffffffffull));
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a1), "r"(b1), "l"(u >> 32));
    hi = r + (v >> 32);
    lo = (v << 32) | (p & 0xffffffffull);
}

// Barrett reduction (Algorithm "Barrett Reduction", L = 63 + Q) of d = (hi,
// lo) < 2^(63+Q) to [0, q).  The exact high word of c1 k leaves the quotient
// short by at most 2 (c4 < 3q); the truncated one (TR, q < 2^61) by at most
// 2 more, so c4 < 5q < 2^64 and three subtractions finish it.
template <bool TR>
__device__ __forceinline__ uint64_t barrett_reduce128v(uint64_t hi, uint64_t lo, uint64_t q,
                                                       uint64_t bk, uint32_t Qm1) {
    const uint64_t c1 = (lo >> Qm1) | (hi << (64 - Qm1));
    const uint64_t c3 = TR ? mulhi64_trunc(c1, bk) : mulhi64_wide(c1, bk);
    uint64_t c4 = lo - c3 * q;
    if (TR) c4 = c4 >= 4 * q ? c4 - 4 * q : c4;
    c4 = c4 >= 2 * q ? c4 - 2 * q : c4;
    return c4 >= q ? c4 - q : c4;
}

// a s mod q in [0, q) for any a < 2^64: the Shoup product, [0, 2q) with the
// exact quotient, [0, 4q) with the truncated one (TR), then subtractions.
template <bool TR>
__device__ __forceinline__ uint64_t tensor_scale64(uint64_t a, const TensorK& c) {
    uint64_t r = shoup_lazy64v<TR ? 3 : 2>(a, c.s, c.sp, c.q, 0 - c.q);
    if (TR) r = r >= 2 * c.q ? r - 2 * c.q : r;
    return r >= c.q ? r - c.q : r;
}

__device__ __forceinline__ uint64_t add_mod_q(uint64_t x, uint64_t e, uint64_t q) {
    const uint64_t t = x + e;   // x, e < q
    return t >= q ? t - q : t;
}

// 32-bit words (q < 2^30): s' = floor(s 2^32 / q) = sp >> 32 and
// k' = floor(2^(31+Q) / q) = bk >> 32 (< 2^32 since q > 2^(Q-1)).  With
// d < 2^(31+Q) (every d here is below 2 q^2 < 2^(2Q+1) <= 2^(31+Q)) the
// quotient c3 = hi32((d >> (Q-1)) k') is short by at most 2, as for 64-bit
// words, and d - c3 q < 3q fits 32 bits.
__device__ __forceinline__ uint32_t barrett_reduce64n(uint64_t d, uint32_t q, uint32_t k32,
                                                      uint32_t Qm1) {
    const uint32_t c3 = __umulhi((uint32_t)(d >> Qm1), k32);
    uint32_t c4 = (uint32_t)d - c3 * q;
    c4 = c4 >= 2 * q ? c4 - 2 * q : c4;
    return c4 >= q ? c4 - q : c4;
}

__device__ __forceinline__ uint32_t tensor_scale32(uint32_t a, uint32_t s, uint32_t sp32,
                                                   uint32_t q) {
    const uint32_t r = shoup_mul_lazy32(a, s, sp32, q);   // [0, 2q) for a < 2^32
    return r >= q ? r - q : r;
}

// a b mod q in [0, q) for a, b < q in the same word classes (the dyadic
// product of the fused polynomial multiply): a b < q^2 is below 2^(63+Q),
// and below 2^(31+Q) on 32-bit words.
template <int Wd>
__device__ __forceinline__ uint64_t mulmod_fused(uint64_t a, uint64_t b, uint64_t q, uint64_t bk,
                                                 uint32_t Qm1) {
    if constexpr (Wd == 0) {
        return barrett_reduce64n((uint64_t)(uint32_t)a * (uint32_t)b, (uint32_t)q,
                                 (uint32_t)(bk >> 32), Qm1);
    } else {
        uint64_t h, l;
        mul_full64(a, b, h, l);
        return barrett_reduce128v<Wd == 1>(h, l, q, bk, Qm1);
    }
}

// Wd: 0 = 32-bit words (q < 2^30, operands < 4q < 2^32), 1 = 64-bit words
// with q < 2^61 (truncated quotients), 2 = 64-bit words, exact quotients.
// a0, a1, b0, b1 < mf q as the forward transform left them; e_k < q.
template <int Wd>
__device__ __forceinline__ void tensor_r3(uint64_t a0, uint64_t a1, uint64_t b0, uint64_t b1,
                                          uint64_t e0, uint64_t e1, uint64_t e2,
                                          const TensorK& c, uint64_t& r0, uint64_t& r1,
                                          uint64_t& r2) {
    b0 = small_mod_rt(b0, c.q, c.mf);
    b1 = small_mod_rt(b1, c.q, c.mf);
    if constexpr (Wd == 0) {
        const uint32_t q = (uint32_t)c.q, s = (uint32_t)c.s, sp = (uint32_t)(c.sp >> 32);
        const uint32_t k = (uint32_t)(c.bk >> 32);
        const uint32_t x0 = tensor_scale32((uint32_t)a0, s, sp, q);
        const uint32_t x1 = tensor_scale32((uint32_t)a1, s, sp, q);
        const uint64_t p0 = (uint64_t)x0 * (uint32_t)b0, p2 = (uint64_t)x1 * (uint32_t)b1;
        const uint64_t p1 = (uint64_t)(x0 + x1) * (uint32_t)(b0 + b1) - p0 - p2;
        r0 = add_mod_q(barrett_reduce64n(p0, q, k, c.Qm1), e0, q);
        r1 = add_mod_q(barrett_reduce64n(p1, q, k, c.Qm1), e1, q);
        r2 = add_mod_q(barrett_reduce64n(p2, q, k, c.Qm1), e2, q);
    } else {
        constexpr bool TR = Wd == 1;
        const uint64_t x0 = tensor_scale64<TR>(a0, c), x1 = tensor_scale64<TR>(a1, c);
        uint64_t h0, l0, h2, l2, h1, l1;
        mul_full64(x0, b0, h0, l0);
        mul_full64(x1, b1, h2, l2);
        mul_full64(x0 + x1, b0 + b1, h1, l1);   // sums < 2q < 2^63
        // (h1, l1) -= (h0, l0) + (h2, l2): a0' b1 + a1' b0 < 2 q^2
        const uint64_t s_lo = l0 + l2;
        const uint64_t s_hi = h0 + h2 + (s_lo < l0 ? 1 : 0);
        h1 = h1 - s_hi - (l1 < s_lo ? 1 : 0);
        l1 = l1 - s_lo;
        r0 = add_mod_q(barrett_reduce128v<TR>(h0, l0, c.q, c.bk, c.Qm1), e0, c.q);
        r1 = add_mod_q(barrett_reduce128v<TR>(h1, l1, c.q, c.bk, c.Qm1), e1, c.q);
        r2 = add_mod_q(barrett_reduce128v<TR>(h2, l2, c.q, c.bk, c.Qm1), e2, c.q);
    }
}

// One r_k (k = 0, 1, 2) in the same arithmetic, for kernels that compute a
// single output: d0 = a0' b0, d2 = a1' b1, d1 = a0' b1 + a1' b0.
template <int Wd>
__device__ __forceinline__ uint64_t tensor_rk(uint32_t k, uint64_t a0, uint64_t a1, uint64_t b0,
                                              uint64_t b1, uint64_t e, const TensorK& c) {
    const uint64_t a = k == 2 ? a1 : a0;                           // the first product's
    const uint64_t b = small_mod_rt(k == 0 ? b0 : b1, c.q, c.mf);  // operands
    const uint64_t bs = small_mod_rt(b0, c.q, c.mf);               // k = 1: a1' b0
    if constexpr (Wd == 0) {
        const uint32_t q = (uint32_t)c.q, s = (uint32_t)c.s, sp = (uint32_t)(c.sp >> 32);
        const uint32_t kk = (uint32_t)(c.bk >> 32);
        uint64_t d = (uint64_t)tensor_scale32((uint32_t)a, s, sp, q) * (uint32_t)b;
        if (k == 1) d += (uint64_t)tensor_scale32((uint32_t)a1, s, sp, q) * (uint32_t)bs;
        return add_mod_q(barrett_reduce64n(d, q, kk, c.Qm1), e, q);
    } else {
        constexpr bool TR = Wd == 1;
        uint64_t h, l;
        mul_full64(tensor_scale64<TR>(a, c), b, h, l);
        if (k == 1) {
            uint64_t h2, l2;
            mul_full64(tensor_scale64<TR>(a1, c), bs, h2, l2);
            l += l2;
            h += h2 + (l < l2 ? 1 : 0);
        }
        return add_mod_q(barrett_reduce128v<TR>(h, l, c.q, c.bk, c.Qm1), e, c.q);
    }
}

}  // namespace hx
