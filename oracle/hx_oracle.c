/*
 * Plain, slow CPU oracle for the negacyclic NTT, the cyclic NTT and the
 * element-wise modular kernels of Intel HEXL (arXiv 2103.16400).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; both receive the same
 * seeded inputs from the separate input-generator module.
 *
 * Every modular product is the paper's naive form (Section 2.1, Listing 1):
 * the exact 128-bit product reduced with the % operator.  Nothing here uses
 * Harvey butterflies, Shoup factors or Barrett reduction: the oracle follows
 * the plain definitions, and the fast method must reach the same values.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *  - Algorithm "Cooley-Tukey Radix-2 NTT" (Section 2.2): the loop header is
 *    read as t = N, m = 1, 2, 4, ... (m doubles), lowercase n meaning N.
 *  - Algorithm "Gentleman-Sande Radix-2 InvNTT": the twiddles are the powers of
 *    psi^-1 in bit-reversed order, indexed h + i.
 *  - The 2N-th root psi, when the caller gives none, is the numerically
 *    smallest primitive 2N-th root of unity mod q.
 *  - psi_rev[0] is never read by the transform; it is stored as 1.
 *  - Element-wise negation b_i = q - a_i (Section 2) is read as (q - a_i) mod q,
 *    so that a_i = 0 gives 0, inside Z_q.
 *  - The cyclic NTT's N-th root omega, when the caller gives none, is the
 *    numerically smallest primitive N-th root of unity mod q.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---- scalar arithmetic (Section 2.1, Listing 1) ------------------------ */

uint64_t oracle_mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * (u128)b) % q);
}

uint64_t oracle_addmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a + (u128)b) % q);
}

uint64_t oracle_submod(uint64_t a, uint64_t b, uint64_t q) {
    a %= q;
    b %= q;
    return a >= b ? a - b : a + (q - b);
}

uint64_t oracle_powmod(uint64_t base, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    base %= q;
    while (e) {
        if (e & 1) r = oracle_mulmod(r, base, q);
        base = oracle_mulmod(base, base, q);
        e >>= 1;
    }
    return r;
}

/* inverse of a mod prime q by Fermat's little theorem */
uint64_t oracle_invmod(uint64_t a, uint64_t q) {
    return oracle_powmod(a, q - 2, q);
}

/* deterministic Miller-Rabin, exact for all 64-bit n with these 12 bases */
int oracle_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n % bases[i] == 0) return n == bases[i];
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = oracle_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int r = 1; r < s; r++) {
            x = oracle_mulmod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/*
 * The numerically smallest primitive 2N-th root of unity mod q (N a power of
 * two, q prime, q = 1 mod 2N).  Since 2N is a power of two, x is a primitive
 * 2N-th root exactly when x^N = -1.  Take g = 2, 3, ... until h = g^((q-1)/2N)
 * satisfies h^N = -1; the primitive roots are then h^(2k+1), k = 0..N-1, and
 * the smallest of them is returned.  Returns 0 if the preconditions fail
 * (N not a power of two, q not prime, q != 1 mod 2N).
 */
uint64_t oracle_min_primitive_root(uint64_t N, uint64_t q) {
    if (N == 0 || (N & (N - 1)) || q < 3 || (q - 1) % (2 * N) != 0) return 0;
    if (!oracle_is_prime(q)) return 0;
    /* h^N = g^((q-1)/2) = -1 exactly when g is a quadratic non-residue; the
       least non-residue of a 64-bit prime is far below this search bound */
    uint64_t h = 0;
    for (uint64_t g = 2; g < q && g < (1ULL << 24); g++) {
        uint64_t c = oracle_powmod(g, (q - 1) / (2 * N), q);
        if (oracle_powmod(c, N, q) == q - 1) { h = c; break; }
    }
    if (h == 0) return 0;
    uint64_t h2 = oracle_mulmod(h, h, q);
    uint64_t x = h, best = h;
    for (uint64_t k = 1; k < N; k++) {
        x = oracle_mulmod(x, h2, q);
        if (x < best) best = x;
    }
    return best;
}

static uint64_t bitrev(uint64_t i, int logn) {
    uint64_t r = 0;
    for (int b = 0; b < logn; b++) { r = (r << 1) | (i & 1); i >>= 1; }
    return r;
}

static int log2u(uint64_t N) {
    int l = 0;
    while ((1ULL << l) < N) l++;
    return l;
}

/* table[k] = root^brv(k) mod q for k = 1..N-1, table[0] = 1 (never read) */
void oracle_bitrev_powers(uint64_t N, uint64_t q, uint64_t root, uint64_t* table) {
    int logn = log2u(N);
    uint64_t* pw = (uint64_t*)malloc(N * sizeof(uint64_t));
    pw[0] = 1 % q;
    for (uint64_t i = 1; i < N; i++) pw[i] = oracle_mulmod(pw[i - 1], root, q);
    for (uint64_t k = 0; k < N; k++) table[k] = pw[bitrev(k, logn)];
    table[0] = 1 % q;
    free(pw);
}

/*
 * Forward negacyclic NTT, Algorithm "Cooley-Tukey Radix-2 NTT" (Section 2.2),
 * in place, standard-order input, bit-reversed output, every butterfly the
 * plain (X0 + W X1 mod q, X0 - W X1 mod q).  Inputs may be any uint64; they
 * are first reduced mod q (the transform depends only on the residues).
 * Output in [0, q).
 */
void oracle_ntt_forward(uint64_t* a, uint64_t N, uint64_t q, const uint64_t* psi_rev) {
    for (uint64_t j = 0; j < N; j++) a[j] %= q;
    uint64_t t = N;
    for (uint64_t m = 1; m < N; m <<= 1) {
        t >>= 1;
        for (uint64_t i = 0; i < m; i++) {
            uint64_t j1 = 2 * i * t;
            uint64_t j2 = j1 + t - 1;
            uint64_t W = psi_rev[m + i];
            for (uint64_t j = j1; j <= j2; j++) {
                uint64_t X0 = a[j];
                uint64_t X1 = a[j + t];
                uint64_t WX1 = oracle_mulmod(W, X1, q);
                a[j] = oracle_addmod(X0, WX1, q);
                a[j + t] = oracle_submod(X0, WX1, q);
            }
        }
    }
}

/*
 * Inverse negacyclic NTT, Algorithm "Gentleman-Sande Radix-2 InvNTT"
 * (Section 2.2): bit-reversed input, standard-order output, butterflies
 * (X0 + X1 mod q, (X0 - X1) W mod q) with W = psiinv_rev[h + i], then the
 * final loop multiplying every coefficient by N^-1 mod q.  Output in [0, q).
 */
void oracle_ntt_inverse(uint64_t* a, uint64_t N, uint64_t q, const uint64_t* psiinv_rev) {
    for (uint64_t j = 0; j < N; j++) a[j] %= q;
    uint64_t t = 1;
    for (uint64_t m = N; m > 1; m >>= 1) {
        uint64_t j1 = 0;
        uint64_t h = m / 2;
        for (uint64_t i = 0; i < h; i++) {
            uint64_t j2 = j1 + t - 1;
            uint64_t W = psiinv_rev[h + i];
            for (uint64_t j = j1; j <= j2; j++) {
                uint64_t X0 = a[j];
                uint64_t X1 = a[j + t];
                a[j] = oracle_addmod(X0, X1, q);
                a[j + t] = oracle_mulmod(oracle_submod(X0, X1, q), W, q);
            }
            j1 += 2 * t;
        }
        t <<= 1;
    }
    uint64_t n_inv = oracle_invmod(N % q, q);
    for (uint64_t j = 0; j < N; j++) a[j] = oracle_mulmod(a[j], n_inv, q);
}

/*
 * Closed form of the bit-reversed negacyclic NTT for selected outputs:
 * out[i] = sum_j a_j psi^((2 brv(i) + 1) j) mod q, i.e. the cyclic NTT of
 * the psi-twisted input (Section 2.2, negative wrapped convolution) read in
 * bit-reversed order.  O(N) per requested index.
 */
void oracle_ntt_forward_direct(const uint64_t* a, uint64_t N, uint64_t q, uint64_t psi,
                               const uint64_t* idx, uint64_t n_idx, uint64_t* out) {
    int logn = log2u(N);
    for (uint64_t k = 0; k < n_idx; k++) {
        uint64_t i = idx[k];
        uint64_t r = oracle_powmod(psi, 2 * bitrev(i, logn) + 1, q);
        uint64_t acc = 0, p = 1 % q;
        for (uint64_t j = 0; j < N; j++) {
            acc = oracle_addmod(acc, oracle_mulmod(a[j] % q, p, q), q);
            p = oracle_mulmod(p, r, q);
        }
        out[k] = acc;
    }
}

/*
 * Negacyclic schoolbook product (Section 2, "vector-vector multiplication"):
 * c_i = sum_{j<=i} a_j b_{i-j} - sum_{j>i} a_j b_{N+i-j} mod q, for selected
 * output indices (all of them when idx is NULL).  O(N) per output.
 */
void oracle_negacyclic_schoolbook(const uint64_t* a, const uint64_t* b, uint64_t N,
                                  uint64_t q, const uint64_t* idx, uint64_t n_idx,
                                  uint64_t* out) {
    uint64_t count = idx ? n_idx : N;
    for (uint64_t k = 0; k < count; k++) {
        uint64_t i = idx ? idx[k] : k;
        uint64_t pos = 0, neg = 0;
        for (uint64_t j = 0; j <= i; j++)
            pos = oracle_addmod(pos, oracle_mulmod(a[j] % q, b[i - j] % q, q), q);
        for (uint64_t j = i + 1; j < N; j++)
            neg = oracle_addmod(neg, oracle_mulmod(a[j] % q, b[N + i - j] % q, q), q);
        out[k] = oracle_submod(pos, neg, q);
    }
}

/* ---- element-wise kernels (Section 2 definitions, Listing 2 semantics) -- */

/* c_i = (a_i + b_i) mod q */
void oracle_eltwise_add_mod(uint64_t* c, const uint64_t* a, const uint64_t* b,
                            uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) c[i] = oracle_addmod(a[i], b[i], q);
}

/* c_i = (a_i - b_i) mod q */
void oracle_eltwise_sub_mod(uint64_t* c, const uint64_t* a, const uint64_t* b,
                            uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) c[i] = oracle_submod(a[i], b[i], q);
}

/* c_i = (a_i * b_i) mod q */
void oracle_eltwise_mult_mod(uint64_t* c, const uint64_t* a, const uint64_t* b,
                             uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) c[i] = oracle_mulmod(a[i], b[i], q);
}

/* c_i = (a_i * s + d_i) mod q; no addend when d is NULL */
void oracle_eltwise_fma_mod(uint64_t* c, const uint64_t* a, uint64_t s, const uint64_t* d,
                            uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) {
        uint64_t p = oracle_mulmod(a[i], s, q);
        c[i] = d ? oracle_addmod(p, d[i], q) : p;
    }
}

/* c_i = (q - a_i) mod q: element-wise negation (Section 2) */
void oracle_eltwise_negate_mod(uint64_t* c, const uint64_t* a, uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) c[i] = oracle_submod(0, a[i], q);
}

/* ---- cyclic NTT (Section 2.2 definitions) ------------------------------- */

/*
 * The numerically smallest primitive N-th root of unity mod q (N a power of
 * two >= 2, q prime, q = 1 mod N): x is primitive exactly when x^(N/2) = -1.
 * Take g = 2, 3, ... until h = g^((q-1)/N) satisfies h^(N/2) = -1; the
 * primitive roots are h^k for odd k < N.  Returns 0 if the preconditions fail.
 */
uint64_t oracle_min_primitive_nth_root(uint64_t N, uint64_t q) {
    if (N < 2 || (N & (N - 1)) || q < 3 || (q - 1) % N != 0) return 0;
    if (!oracle_is_prime(q)) return 0;
    uint64_t h = 0;
    for (uint64_t g = 2; g < q && g < (1ULL << 24); g++) {
        uint64_t c = oracle_powmod(g, (q - 1) / N, q);
        if (oracle_powmod(c, N / 2, q) == q - 1) { h = c; break; }
    }
    if (h == 0) return 0;
    uint64_t h2 = oracle_mulmod(h, h, q);
    uint64_t x = h, best = h;
    for (uint64_t k = 1; k < N / 2; k++) {
        x = oracle_mulmod(x, h2, q);
        if (x < best) best = x;
    }
    return best;
}

/*
 * Forward cyclic NTT by its definition, natural order, for selected outputs:
 * out[k] = sum_j a_j omega^(i j) mod q with i = idx[k].  O(N) per output.
 */
void oracle_cyclic_ntt_direct(const uint64_t* a, uint64_t N, uint64_t q, uint64_t omega,
                              const uint64_t* idx, uint64_t n_idx, uint64_t* out) {
    for (uint64_t k = 0; k < n_idx; k++) {
        uint64_t r = oracle_powmod(omega, idx[k] % N, q);
        uint64_t acc = 0, p = 1 % q;
        for (uint64_t j = 0; j < N; j++) {
            acc = oracle_addmod(acc, oracle_mulmod(a[j] % q, p, q), q);
            p = oracle_mulmod(p, r, q);
        }
        out[k] = acc;
    }
}

/*
 * Inverse cyclic NTT by its definition, natural order, all outputs:
 * b_i = N^-1 sum_j x_j omega^(-i j) mod q.  O(N^2).
 */
void oracle_cyclic_intt_direct(const uint64_t* x, uint64_t N, uint64_t q, uint64_t omega,
                               uint64_t* b) {
    uint64_t winv = oracle_invmod(omega, q), ninv = oracle_invmod(N % q, q);
    for (uint64_t i = 0; i < N; i++) {
        uint64_t r = oracle_powmod(winv, i, q);
        uint64_t acc = 0, p = 1 % q;
        for (uint64_t j = 0; j < N; j++) {
            acc = oracle_addmod(acc, oracle_mulmod(x[j] % q, p, q), q);
            p = oracle_mulmod(p, r, q);
        }
        b[i] = oracle_mulmod(acc, ninv, q);
    }
}

/*
 * Cyclic schoolbook product in Z_q[X] / (X^N - 1), selected outputs (all
 * when idx is NULL): c_i = sum_j a_j b_((i - j) mod N) mod q.  O(N) each.
 */
void oracle_cyclic_schoolbook(const uint64_t* a, const uint64_t* b, uint64_t N, uint64_t q,
                              const uint64_t* idx, uint64_t n_idx, uint64_t* out) {
    uint64_t count = idx ? n_idx : N;
    for (uint64_t k = 0; k < count; k++) {
        uint64_t i = idx ? idx[k] : k;
        uint64_t acc = 0;
        for (uint64_t j = 0; j < N; j++)
            acc = oracle_addmod(acc, oracle_mulmod(a[j] % q, b[(i + N - j) % N] % q, q), q);
        out[k] = acc;
    }
}
