/*
 * hexgpu -- negacyclic NTT and element-wise modular arithmetic over RNS limbs
 * on one NVIDIA GB300 (sm_103a).  C ABI.
 *
 * The operations are those of Intel HEXL (arXiv 2103.16400): the forward and
 * inverse negacyclic number-theoretic transform over Z_q[X]/(X^N + 1)
 * (Section 2.2: Cooley-Tukey forward with bit-reversed output, Gentleman-Sande
 * inverse with N^-1 scaling, Harvey lazy butterflies, Shoup twiddle factors)
 * and the element-wise kernels EltwiseAddMod, EltwiseMultMod, EltwiseFMAMod
 * (Section 3, free-function API), batched over polynomials and RNS limbs
 * (Section 4 describes the RNS form, in which limbs are independent).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Layout.    A batch of polynomials is a dense uint64 array
 *             [n_polys][n_limbs][N]: limb l of polynomial p starts at
 *             ptr + (p * n_limbs + l) * N.  Element-wise calls use the same
 *             layout with a row length n instead of N.
 *  Memory.    Arguments named d_* are device pointers that the caller owns
 *             (for example torch tensor storage), 16-byte aligned.  Arguments
 *             named h_* are host pointers, read during the call only.
 *             A result may alias its operand exactly (in-place operation);
 *             partial overlap is rejected.
 *  Streams.   Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy
 *             default stream) and the call returns without waiting for it.
 *             Errors detected on the host are returned before anything is
 *             enqueued; launch errors are returned as HX_ERR_CUDA.
 *  Moduli.    q must be prime with q = 1 mod 2N for the transforms
 *             (Section 2: q = 1 mod 2N), and below 2^62 (the Harvey
 *             butterflies require q < beta/4 with beta = 2^64).  Limbs with
 *             q < 2^30 run on 32-bit words (beta = 2^32).
 *  Lazy ranges. input_mod_factor k promises every input value is in [0, k q);
 *             output_mod_factor k returns values in [0, k q) that are
 *             congruent to the exact result (Section 3, NTT class API).
 *             Inputs outside the promised range give undefined results, as
 *             in the paper.
 *  Threads.   Calls may be made from several host threads; a plan may be used
 *             by several streams at once but destroyed only when idle.
 *  Errors.    Every call returns HX_OK (0) or a negative hx_status;
 *             hx_strerror() names it.
 */
#ifndef HEXGPU_H
#define HEXGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* hx_stream_t; /* same type as cudaStream_t */
typedef struct hx_plan_s* hx_plan_t;
typedef struct hx_batch_s* hx_batch_t;

typedef enum hx_status {
    HX_OK = 0,
    HX_ERR_NULL = -1,         /* a required pointer is NULL */
    HX_ERR_ALIGN = -2,        /* a device pointer is not 16-byte aligned */
    HX_ERR_DEGREE = -3,       /* N is not a power of two in [2^10, 2^17] */
    HX_ERR_MODULUS = -4,      /* q not prime, q != 1 mod 2N, or q out of range */
    HX_ERR_ROOT = -5,         /* a supplied root is not a primitive 2N-th root */
    HX_ERR_MOD_FACTOR = -6,   /* input/output mod factor not allowed */
    HX_ERR_CUDA = -7,         /* a CUDA runtime call failed */
    HX_ERR_ARG = -8,          /* another argument is out of range */
    HX_ERR_OVERLAP = -9,      /* result and operand partially overlap */
    HX_ERR_TIMEOUT = -10,     /* a device-side wait gave up */
    HX_ERR_NOMEM = -11,       /* device or host allocation failed */
    HX_ERR_CAPACITY = -12     /* request exceeds a fixed scratch capacity */
} hx_status;

const char* hx_strerror(int status);

/* Version of this ABI; bumps on any incompatible change. */
int hx_abi_version(void);

/* --------------------------------------------------------------------- plan
 * A plan owns, in device memory, the per-limb tables that the paper's NTT
 * class precomputes at construction (Section 3, "The NTT class performs
 * pre-computation"): psi_rev (powers of psi in bit-reversed order, the
 * Cooley-Tukey twiddles), psi^-1_rev (the Gentleman-Sande twiddles), the
 * Shoup factor W' = floor(W beta / q) of each, N^-1 and its Shoup factor.
 *
 * hx_plan_create(out, N, h_moduli, n_limbs, h_roots)
 *   N         transform length, a power of two in [2^10, 2^17].
 *   h_moduli  host array of n_limbs primes, each q = 1 mod 2N and q < 2^62.
 *   n_limbs   1 .. 4096.
 *   h_roots   host array of n_limbs primitive 2N-th roots of unity (psi, one
 *             per modulus) or NULL.  When NULL, psi is the numerically
 *             smallest primitive 2N-th root of unity mod q (the paper leaves
 *             psi open when none is given).
 *   *out      receives the plan.  The plan allocates 32*N bytes of device
 *             memory per limb on the current device, and is valid on that
 *             device only.
 *   Errors: HX_ERR_NULL, HX_ERR_DEGREE, HX_ERR_MODULUS, HX_ERR_ROOT,
 *   HX_ERR_ARG, HX_ERR_NOMEM, HX_ERR_CUDA.
 */
int hx_plan_create(hx_plan_t* out, uint64_t N, const uint64_t* h_moduli, uint32_t n_limbs,
                   const uint64_t* h_roots);

/* hx_plan_create_cyclic: a plan for the cyclic NTT of Section 2.2,
 *   NTT(a)_i = sum_j a_j omega^(i j) mod q, omega a primitive N-th root of
 *   unity, and its inverse InvNTT(x)_i = N^-1 sum_j x_j omega^(-i j) mod q.
 *   hx_ntt_forward / hx_ntt_inverse (and the ragged batches) on this plan
 *   give these transforms with the same bit-reversed output (forward) and
 *   input (inverse) order, mod factors and errors as for negacyclic plans,
 *   and hx_poly_mul gives the product in Z_q[X] / (X^N - 1).
 *   h_moduli  primes q = 1 mod N, q < 2^62.
 *   h_roots   n_limbs primitive N-th roots omega, or NULL for the
 *             numerically smallest one per modulus; hx_plan_roots returns
 *             omega for these plans.
 *   Other arguments, memory and errors as hx_plan_create. */
int hx_plan_create_cyclic(hx_plan_t* out, uint64_t N, const uint64_t* h_moduli,
                          uint32_t n_limbs, const uint64_t* h_roots);
int hx_plan_destroy(hx_plan_t plan);

/* Copies the plan's root per limb (psi; omega for cyclic plans) into
 * h_roots_out[n_limbs]. */
int hx_plan_roots(hx_plan_t plan, uint64_t* h_roots_out);

/* Plan shape: N, limb count and the device bytes the plan holds. */
int hx_plan_info(hx_plan_t plan, uint64_t* N, uint32_t* n_limbs, uint64_t* device_bytes);

/* Kernel schedule of the plan's transforms -- the knob the autotuner turns;
 * any valid schedule gives identical results, only speed differs (the paper
 * suggests choosing implementations by trials, Section 3.2).  npass is 1 or
 * 2; params holds seven int32 per pass, in stage order:
 *   {s0, K, logGb, logGc, logR, pipe, np}
 * pass covers stages [s0, s0 + K) of the log2 N stages; a tile is
 * 2^logGb x 2^K x 2^logGc elements (top-index values x stage bits x
 * low-index values); 2^logR elements per thread; pipe = 1 selects the
 * persistent double-buffered kernel, pipe = 2 the per-tile kernel that first
 * copies the tile's twiddle pairs into shared memory (pipe = 0: per-tile,
 * twiddles read through the read-only cache); np (1 or 2) is the number of
 * polynomials each thread transforms with one set of twiddle registers.
 * pipe = 3 on both passes of a two-pass schedule,
 *   {0, K1, 0, logGc, logR, 3, 1}, {K1, K2, logGb, 0, logR, 3, 1}
 * with K2 - logGc = K1 - logGb = c in [1, 4], fuses them into one launch of
 * thread-block clusters of 2^c CTAs per limb-transform: each CTA keeps N/2^c
 * coefficients in shared memory, the column stages and the row stages run
 * there, and the CTAs exchange between the two through distributed shared
 * memory, so every coefficient crosses HBM once each way (N in [2^14, 2^17]).
 * hx_plan_set_schedule returns HX_ERR_ARG for a schedule the library cannot
 * run (stages not covering [0, log2 N), a kernel not in the menu, tile too
 * large, a cluster shape the device cannot make resident).  `direction` selects the forward (1) or inverse (2) transform's
 * schedule, or both (3, set only); the inverse runs the same passes in
 * reverse order.  hx_plan_get_schedule writes 14 int32 (the unused second
 * pass zeroed). */
int hx_plan_set_schedule(hx_plan_t plan, uint32_t direction, uint32_t npass,
                         const int32_t* params);
int hx_plan_get_schedule(hx_plan_t plan, uint32_t direction, uint32_t* npass, int32_t* params);

/* ----------------------------------------------------------------- transforms
 * hx_ntt_forward: forward negacyclic NTT of every limb of n_polys
 *   polynomials (Section 2.2, Algorithm "Cooley-Tukey Radix-2 NTT" with the
 *   Harvey butterfly): d_result[i] = sum_j d_operand[j] psi^((2 brv(i)+1) j)
 *   mod q, output in bit-reversed order.
 *   d_operand, d_result: [n_polys][plan n_limbs][N] uint64, equal or disjoint.
 *   input_mod_factor in {1, 2, 4}; output_mod_factor in {1, 4}.
 *
 * hx_ntt_inverse: inverse negacyclic NTT (Algorithm "Gentleman-Sande Radix-2
 *   InvNTT" with the Harvey inverse butterfly and the N^-1 scaling folded
 *   into the last stage): bit-reversed input, standard-order output.
 *   input_mod_factor in {1, 2}; output_mod_factor in {1, 2}.
 *
 * Both enqueue the transform on `stream`.  Errors: HX_ERR_NULL, HX_ERR_ALIGN,
 * HX_ERR_ARG (n_polys == 0), HX_ERR_MOD_FACTOR, HX_ERR_OVERLAP, HX_ERR_CUDA.
 */
int hx_ntt_forward(hx_plan_t plan, uint64_t* d_result, const uint64_t* d_operand,
                   uint32_t n_polys, uint32_t input_mod_factor, uint32_t output_mod_factor,
                   hx_stream_t stream);
int hx_ntt_inverse(hx_plan_t plan, uint64_t* d_result, const uint64_t* d_operand,
                   uint32_t n_polys, uint32_t input_mod_factor, uint32_t output_mod_factor,
                   hx_stream_t stream);

/* In-place transforms of one polynomial's n_limbs limbs ([n_limbs][N] at
 * d_ptr), the (ptr, N, q, n_limbs, input_mod_factor, output_mod_factor) form
 * of the problem statement.  The plan for (N, moduli) is built on first use
 * and cached (the first call for a new modulus set is therefore slow and
 * allocates; call it once outside any stream capture).  Same errors as above
 * plus those of hx_plan_create. */
int hx_ntt_forward_raw(uint64_t* d_ptr, uint64_t N, const uint64_t* h_moduli, uint32_t n_limbs,
                       uint32_t input_mod_factor, uint32_t output_mod_factor,
                       hx_stream_t stream);
int hx_ntt_inverse_raw(uint64_t* d_ptr, uint64_t N, const uint64_t* h_moduli, uint32_t n_limbs,
                       uint32_t input_mod_factor, uint32_t output_mod_factor,
                       hx_stream_t stream);

/* --------------------------------------------------------------- element-wise
 * All take rows of n elements in the [n_polys][n_limbs][n] layout; row
 * (p, l) is reduced modulo h_moduli[l].  n >= 1 (any n: no multiple-of-8
 * requirement, Section 3.3 handles the N mod 8 tail the same way).
 *
 * hx_eltwise_add_mod: r = (a + b) mod q; a, b in [0, q); q in [2, 2^63 - 1]
 *   (Section 3, EltwiseAddMod).
 * hx_eltwise_sub_mod: r = (a - b) mod q; a, b in [0, q); q in [2, 2^63 - 1].
 * hx_eltwise_negate_mod: r = (q - a) mod q (Section 2, element-wise
 *   negation b_i = q - a_i, taken mod q so that 0 maps to 0); a in [0, q);
 *   q in [2, 2^63 - 1]; r may equal a.
 * hx_eltwise_mult_mod: r = (a * b) mod q, a and b in [0, k q) for
 *   k = input_mod_factor in {1, 2, 4}; q in [2, 2^62) with k q < 2^63
 *   (Section 3.3, Algorithm "VectorVectorModMulAVX512Int": Barrett reduction
 *   with Q = bitlen(q), L = 63 + Q).
 * hx_eltwise_fma_mod: r = (a * s_l + d) mod q with one scalar s_l in [0, q)
 *   per limb (h_scalars, host) and an optional addend d (NULL: none);
 *   a, d in [0, k q), k = input_mod_factor in {1, 2, 4, 8}; q in [2, 2^61 - 1]
 *   (Section 3.3, Algorithm "EltwiseFMAModAVX512").
 * Outputs are in [0, q).  Errors: HX_ERR_NULL, HX_ERR_ALIGN, HX_ERR_ARG,
 * HX_ERR_MODULUS, HX_ERR_MOD_FACTOR, HX_ERR_OVERLAP, HX_ERR_CUDA.
 */
int hx_eltwise_add_mod(uint64_t* d_result, const uint64_t* d_a, const uint64_t* d_b, uint64_t n,
                       const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys,
                       hx_stream_t stream);
int hx_eltwise_sub_mod(uint64_t* d_result, const uint64_t* d_a, const uint64_t* d_b, uint64_t n,
                       const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys,
                       hx_stream_t stream);
int hx_eltwise_negate_mod(uint64_t* d_result, const uint64_t* d_a, uint64_t n,
                          const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys,
                          hx_stream_t stream);
int hx_eltwise_mult_mod(uint64_t* d_result, const uint64_t* d_a, const uint64_t* d_b, uint64_t n,
                        const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys,
                        uint32_t input_mod_factor, hx_stream_t stream);
int hx_eltwise_fma_mod(uint64_t* d_result, const uint64_t* d_a, const uint64_t* h_scalars,
                       const uint64_t* d_addend, uint64_t n, const uint64_t* h_moduli,
                       uint32_t n_limbs, uint32_t n_polys, uint32_t input_mod_factor,
                       hx_stream_t stream);

/* --------------------------------------------------------------- compositions
 * hx_poly_mul: negacyclic product r = a * b in R_q per limb, composed as in
 *   the paper's Listing 4: forward NTT of a and of b in place with output in
 *   [0, 4q), EltwiseMultMod with input_mod_factor 4, inverse NTT to [0, q).
 *   When the plan's inverse schedule starts with a per-tile row pass (or a
 *   single pass), the element-wise product runs inside that pass (the
 *   kernel-sequence fusion the paper's Conclusion points to): the product
 *   never goes to HBM and one launch disappears; the result is the same.
 *   d_a and d_b are overwritten with their transforms; d_result may equal
 *   d_a.  All [n_polys][plan n_limbs][N].
 *
 * hx_ciphertext_tensor: product of two degree-1 ciphertexts (a0, a1) and
 *   (b0, b1) in coefficient form, followed by a scaled accumulation:
 *     A_i, B_i = forward NTT of a_i, b_i (in place, output in [0, 4q))
 *     d0 = A0 B0,  d1 = A0 B1 + A1 B0,  d2 = A1 B1   (element-wise mod q)
 *     r_k = d_k * s_l + e_k mod q                    (EltwiseFMAMod)
 *     out_k = inverse NTT of r_k, in [0, q).
 *   The products, the sum, the scaling and the inverse transform run as
 *   hx_tensor_fma_inverse below; all steps are enqueued on `stream`.  e_k
 *   are in [0, q) (NTT domain); h_scalars holds one s_l in [0, q) per limb.
 *   The four inputs are overwritten with their transforms; out_k must not
 *   alias any input.
 *
 * hx_tensor_fma_inverse: the NTT-domain half of hx_ciphertext_tensor --
 *   from forward transforms A0, A1, B0, B1 in [0, input_mod_factor q)
 *   (input_mod_factor in {1, 2, 4}) and addends e_k in [0, q):
 *     r_k = d_k s_l + e_k mod q (d_k as above),  out_k = inverse NTT of r_k,
 *   in [0, q).  When A0..B1 lie back to back from A0 ([4][n_polys][limbs][N]),
 *   e0..e2 from e0 and out0..out2 from out0 ([3][n_polys][limbs][N]), and
 *   the plan's inverse schedule starts with a per-tile pass (pipe 0 or 2),
 *   the element-wise step runs inside the first pass of the inverse
 *   transform, so the r_k are never written to device memory (cross-kernel
 *   fusion, the direction Section 5 names); otherwise it runs as
 *   hx_dyadic_tensor_fma followed by hx_ntt_inverse.  Both give the same
 *   bits.  Moduli must be < 2^61; out_k must not alias any input.  Errors:
 *   HX_ERR_NULL, HX_ERR_ARG, HX_ERR_MOD_FACTOR, HX_ERR_MODULUS, HX_ERR_ALIGN,
 *   HX_ERR_OVERLAP, HX_ERR_CUDA.
 */
int hx_poly_mul(hx_plan_t plan, uint64_t* d_result, uint64_t* d_a, uint64_t* d_b,
                uint32_t n_polys, hx_stream_t stream);

/* hx_dyadic_inverse: d_result = InvNTT(d_A . d_B), the second half of the
 *   paper's Listing 4 on spectra the caller already holds: EltwiseMultMod of
 *   the forward outputs d_A and d_B (both below input_mod_factor q,
 *   input_mod_factor 1, 2 or 4; q below 2^62 and 4q below 2^64) followed by
 *   the inverse NTT to [0, q).  The product runs inside the inverse's first
 *   pass when the plan's inverse schedule starts with a per-tile row pass,
 *   else as a separate element-wise pass into d_result first.  All
 *   [n_polys][plan n_limbs][N]; d_A and d_B are only read; d_result may
 *   equal d_A or d_B, or be disjoint from both.
 *   Errors: HX_ERR_NULL, HX_ERR_ALIGN, HX_ERR_ARG, HX_ERR_MOD_FACTOR,
 *   HX_ERR_OVERLAP, HX_ERR_CUDA. */
int hx_dyadic_inverse(hx_plan_t plan, uint64_t* d_result, const uint64_t* d_A,
                      const uint64_t* d_B, uint32_t n_polys, uint32_t input_mod_factor,
                      hx_stream_t stream);
int hx_ciphertext_tensor(hx_plan_t plan, uint64_t* d_out0, uint64_t* d_out1, uint64_t* d_out2,
                         uint64_t* d_a0, uint64_t* d_a1, uint64_t* d_b0, uint64_t* d_b1,
                         const uint64_t* h_scalars, const uint64_t* d_e0, const uint64_t* d_e1,
                         const uint64_t* d_e2, uint32_t n_polys, hx_stream_t stream);

int hx_tensor_fma_inverse(hx_plan_t plan, uint64_t* d_out0, uint64_t* d_out1, uint64_t* d_out2,
                          const uint64_t* d_A0, const uint64_t* d_A1, const uint64_t* d_B0,
                          const uint64_t* d_B1, const uint64_t* h_scalars, const uint64_t* d_e0,
                          const uint64_t* d_e1, const uint64_t* d_e2, uint32_t n_polys,
                          uint32_t input_mod_factor, hx_stream_t stream);

/* hx_poly_product: d_result = d_a * d_b in R_q = Z_q[X]/(X^N + 1) (the paper's
 *   Listing 4: forward NTT of both, EltwiseMultMod with input_mod_factor 4,
 *   inverse NTT to [0, q)) with the operands kept: d_a, d_b in [0, q), only
 *   read; d_work ([2][n_polys][limbs][N]) is scratch the caller provides,
 *   apart from d_a, d_b and d_result; d_result may equal d_a or d_b.  When
 *   the plan's forward and inverse schedules are both two-pass over the same
 *   stages with 8 elements a thread in their row passes, the call is four
 *   launches: the forward's column pass of a and of b, one kernel that runs
 *   the forward's row stages on both, the dyadic product and the inverse's
 *   row stages (in the inverse's row tiles) with the spectra in shared
 *   memory, and the inverse's column pass; otherwise hx_ntt_forward of each
 *   into d_work followed by hx_dyadic_inverse.  Both give the same bits.
 *   Moduli below 2^62.  All [n_polys][plan n_limbs][N], 16-byte aligned.
 *   Errors: HX_ERR_NULL, HX_ERR_ARG, HX_ERR_ALIGN, HX_ERR_OVERLAP, HX_ERR_CUDA. */
int hx_poly_product(hx_plan_t plan, uint64_t* d_result, const uint64_t* d_a, const uint64_t* d_b,
                    uint64_t* d_work, uint32_t n_polys, hx_stream_t stream);

/* hx_ciphertext_step: the whole ciphertext tensor product (the computation of
 *   hx_ciphertext_tensor) on operands laid out back to back, with the
 *   operands kept: d_in holds a0 | a1 | b0 | b1 ([4][n_ct][limbs][N], in
 *   [0, q)), d_e the addends e0 | e1 | e2 ([3][n_ct][limbs][N], in [0, q), NTT
 *   domain), h_scalars one s_l in [0, q) per limb (host); d_result receives
 *   out0 | out1 | out2 ([3][n_ct][limbs][N], in [0, q)):
 *     out_k = InvNTT(d_k s_l + e_k),  d0 = A0 B0, d1 = A0 B1 + A1 B0,
 *     d2 = A1 B1,  A_i, B_i = NTT(a_i, b_i)           (Section 2.2, Listing 4)
 *   d_work ([4][n_ct][limbs][N]) is scratch the caller provides; it may equal
 *   d_in (the operands are then overwritten).  When the plan's forward and
 *   inverse schedules are both two-pass with row passes over the same stages
 *   (8 elements a thread, 6..9 row stages; the inverse's row tile is used for
 *   both), the call is three launches: the forward's column
 *   pass, one kernel that runs the forward's row stages on the four operands,
 *   the tensor step and the inverse's row stages on the three outputs with
 *   the spectra kept in shared memory (they never reach HBM), and the
 *   inverse's column pass; otherwise hx_ntt_forward into d_work followed by
 *   hx_tensor_fma_inverse.  Both give the same bits.  Moduli must be < 2^61;
 *   d_result must not overlap d_in, d_work or d_e.  Pointers 16-byte aligned.
 *   Errors: HX_ERR_NULL, HX_ERR_ARG, HX_ERR_MODULUS, HX_ERR_ALIGN,
 *   HX_ERR_OVERLAP, HX_ERR_CUDA. */
int hx_ciphertext_step(hx_plan_t plan, uint64_t* d_result, const uint64_t* d_in,
                       uint64_t* d_work, const uint64_t* h_scalars, const uint64_t* d_e,
                       uint32_t n_ct, hx_stream_t stream);

/* Fused element-wise part of hx_ciphertext_tensor on its own: reads A0, A1,
 * B0, B1 in [0, input_mod_factor q) (input_mod_factor in {1, 2, 4}) and e_k
 * in [0, q), writes r_k in [0, q).  Rows of n elements, [n_polys][n_limbs][n]. */
int hx_dyadic_tensor_fma(uint64_t* d_r0, uint64_t* d_r1, uint64_t* d_r2, const uint64_t* d_A0,
                         const uint64_t* d_A1, const uint64_t* d_B0, const uint64_t* d_B1,
                         const uint64_t* h_scalars, const uint64_t* d_e0, const uint64_t* d_e1,
                         const uint64_t* d_e2, uint64_t n, const uint64_t* h_moduli,
                         uint32_t n_limbs, uint32_t n_polys, uint32_t input_mod_factor,
                         hx_stream_t stream);

/* -------------------------------------------------------------- ragged batches
 * Many transforms of different N and modulus sets in one replay: the
 * paper's per-call NTT (Section 3) is too small to fill a GPU by itself
 * (Section 4 notes the offload problem), so a batch gathers every
 * (polynomial, limb) transform of every item into one tile list and runs it
 * as one persistent kernel per pass, captured once into a CUDA graph.
 *
 * hx_ragged_item: one group of polynomials sharing a plan.
 *   plan     the plan (N and moduli) of these polynomials
 *   d_in     device operand [n_polys][plan n_limbs][N]
 *   d_out    device result, same shape; equal to d_in or disjoint
 *   n_polys  >= 1
 *
 * hx_batch_create(out, h_items, n_items, direction, input_mod_factor,
 *                 output_mod_factor)
 *   h_items  host array of n_items items (read during the call only); the
 *            plans and device buffers must outlive the batch.
 *   direction 1 = forward (input_mod_factor 1/2/4, output 1/4),
 *             2 = inverse (input 1/2, output 1/2); the same semantics as
 *             hx_ntt_forward / hx_ntt_inverse per transform.
 *   Allocates the tile list (32 bytes per 2048-element tile) and two work
 *   counters in device memory on the current device, and instantiates the
 *   graph.  Errors: HX_ERR_NULL, HX_ERR_ALIGN, HX_ERR_ARG, HX_ERR_MOD_FACTOR,
 *   HX_ERR_OVERLAP, HX_ERR_NOMEM, HX_ERR_CUDA.
 * hx_batch_run: enqueues one replay of the whole batch on `stream` (one
 *   graph launch: counter reset, then one or two persistent passes).
 *   Replays on different streams must not overlap in time (they share the
 *   counters).
 * hx_batch_info: transforms, tiles and kernel launches per replay.
 *
 * hx_ragged_set_split(log2_n, k1) / hx_ragged_get_split(log2_n, &k1): the
 *   pass shapes of ragged transforms of N = 2^log2_n (12 <= log2_n <= 17): a
 *   column pass over the first k1 stages then a row pass over the other
 *   log2_n - k1, both on 2048-element tiles; k1 in [5, 9] with
 *   6 <= log2_n - k1 <= 11.  Every split gives the same results (it is the
 *   knob the autotuner turns -- the paper's "choose by trials", Section
 *   3.2).  The setting is process-wide and read when the tile lists are
 *   written: by hx_batch_create (a batch keeps the shapes it was created
 *   with), hx_batch_run_static, hx_ntt_ragged and hx_polymul_ragged.
 *   Errors: HX_ERR_ARG (split or log2_n outside the menu), HX_ERR_NULL.
 */
typedef struct hx_ragged_item {
    hx_plan_t plan;
    const uint64_t* d_in;
    uint64_t* d_out;
    uint32_t n_polys;
    uint32_t reserved;
} hx_ragged_item;

int hx_ragged_set_split(uint32_t log2_n, uint32_t k1);
int hx_ragged_get_split(uint32_t log2_n, uint32_t* k1);
int hx_batch_create(hx_batch_t* out, const hx_ragged_item* h_items, uint32_t n_items,
                    uint32_t direction, uint32_t input_mod_factor, uint32_t output_mod_factor);
int hx_batch_run(hx_batch_t batch, hx_stream_t stream);
int hx_batch_info(hx_batch_t batch, uint64_t* limb_transforms, uint64_t* tiles,
                  uint32_t* launches);
int hx_batch_destroy(hx_batch_t batch);

/* hx_batch_run_static: runs the same ragged set of transforms once, like
 * hx_batch_create + hx_batch_run + hx_batch_destroy, but without allocating
 * any device memory.  The paper has no counterpart; it exists for callers
 * that cannot call cudaMalloc where they need the transforms -- a serving
 * loop that admits work against a fixed device-memory budget, an application
 * whose own memory pool owns the whole GPU, or a latency-critical path that
 * cannot absorb the device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * The work counters and the tile list live in one fixed 4 MiB array compiled
 * into the library; every GPU that loads the library holds that array until
 * the process exits.  A request may hold at most 131064 tiles (one tile per
 * 2048 coefficients per pass: N <= 2^11 takes one pass, larger N two);
 * larger requests are refused with HX_ERR_CAPACITY before anything is
 * enqueued.  Arguments, semantics and the other errors are those of
 * hx_batch_create; the tile list is copied from host memory on `stream`
 * and the kernels are enqueued there (no graph).
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any
 * stream capture.  Like the plans' device tables, the cached address
 * belongs to the device's context as it was at that call: after a device
 * reset (cudaDeviceReset, or the primary context torn down and made anew)
 * neither may be used again in this process.  All calls share the one array and it keeps the last
 * call's contents (the counters are re-zeroed on `stream` by each call):
 * calls whose work overlaps on the GPU -- on different streams, or on one
 * device from several host threads without ordering -- race on it. */
int hx_batch_run_static(const hx_ragged_item* h_items, uint32_t n_items, uint32_t direction,
                        uint32_t input_mod_factor, uint32_t output_mod_factor,
                        hx_stream_t stream);

/* hx_ntt_ragged: the same single run of a ragged set of transforms (Algorithm
 * CT forward or GS inverse with N^-1, per item's plan; direction 1 or 2 and
 * the mod factors as for hx_batch_create), with the work counters and the
 * tile list in a caller-owned device workspace instead of the library's
 * fixed array -- the serving primitive for transform requests: calls on
 * different streams, each with its own workspace, may overlap.
 *   d_workspace: device memory, 256-byte aligned, at least the size
 *   hx_ntt_ragged_workspace reports for the same items (256 bytes plus 32
 *   bytes per tile); reusable by calls ordered on one stream.  The tile list
 *   is written on the host into the library's pooled page-locked staging
 *   (as for hx_polymul_ragged) and uploaded on `stream`; two kernels run on
 *   `stream` (one for N <= 2^11 alone).  The call returns without waiting.
 *   Errors: those of hx_batch_create, HX_ERR_ALIGN (workspace),
 *   HX_ERR_CAPACITY (workspace too small), HX_ERR_NOMEM (no staging). */
int hx_ntt_ragged_workspace(const hx_ragged_item* h_items, uint32_t n_items, uint64_t* bytes);
int hx_ntt_ragged(const hx_ragged_item* h_items, uint32_t n_items, uint32_t direction,
                  uint32_t input_mod_factor, uint32_t output_mod_factor, void* d_workspace,
                  uint64_t workspace_bytes, hx_stream_t stream);

/* --------------------------------------------- ragged products (serving primitive)
 * hx_polymul_ragged: for every item, d_result = d_a * d_b in R_q for each
 *   polynomial and limb of the item's plan, composed as the paper's Listing 4
 *   (forward NTT of both operands with output range [0, 4q), EltwiseMultMod
 *   with input_mod_factor 4, inverse NTT to [0, q)).  Items may differ in N
 *   and moduli (every modulus below 2^61).  Operands are read, never
 *   written: the forward transforms go out of place into the workspace and
 *   the inverse writes the result.  The whole set runs as four kernels on
 *   `stream`: two forward passes, then the inverse's two passes, the first
 *   of which computes the element-wise product while it stages each tile
 *   (the product never goes to HBM).
 *   hx_polymul_item: plan; d_a, d_b, d_result: device [n_polys][limbs][N]
 *   (d_result may equal d_a or d_b); n_polys >= 1.
 *   d_workspace: caller-owned device memory, 256-byte aligned, at least the
 *   size hx_polymul_ragged_workspace reports (twice the operand size plus
 *   32 to 48 bytes per tile and pass); it holds the spectra, the tile lists and the work
 *   counters, so the library allocates no device memory.  A workspace may be
 *   reused by calls ordered on one stream, not by concurrent ones.  The tile
 *   lists are written on the host into page-locked staging buffers that the
 *   library keeps (a pool grown on demand, each reused once its upload has
 *   completed, held for the life of the process) and uploaded asynchronously
 *   on `stream`; the call returns without waiting for the GPU.
 *   Errors: HX_ERR_NULL, HX_ERR_ALIGN, HX_ERR_ARG, HX_ERR_MODULUS,
 *   HX_ERR_CAPACITY (workspace too small), HX_ERR_NOMEM (no page-locked
 *   staging), HX_ERR_CUDA. */
typedef struct hx_polymul_item {
    hx_plan_t plan;
    const uint64_t* d_a;
    const uint64_t* d_b;
    uint64_t* d_result;
    uint32_t n_polys;
    uint32_t reserved;
} hx_polymul_item;

int hx_polymul_ragged_workspace(const hx_polymul_item* h_items, uint32_t n_items,
                                uint64_t* bytes);
int hx_polymul_ragged(const hx_polymul_item* h_items, uint32_t n_items, void* d_workspace,
                      uint64_t workspace_bytes, hx_stream_t stream);

/* ---------------------------------------------------------------- measurement
 * Support for the benchmark; the paper has no counterpart.
 *
 * hx_launch_count: number of CUDA kernels this library has launched in this
 *   process (all entry points, all devices), for launch accounting.
 * hx_probe_int_mul_rate: runs a grid of 8 blocks of 256 threads per SM in
 *   which every thread executes `iters` x 16 instructions of one 32-bit
 *   integer multiply form in 8 independent dependency chains -- kind 0:
 *   mad.lo.u32, kind 1: mad.hi.u32, kind 2: mad.wide.u32, kind 3: lo and hi
 *   alternating -- and returns the achieved rate in *ops_per_s (and the
 *   kernel time in *ms if not NULL): the integer-multiply roofline of this
 *   GPU at its current clocks.  Synchronises `stream`.
 * hx_probe_butterfly_rate: the same grid running Harvey butterflies for
 *   modulus q on register-resident data (4 per thread per iteration);
 *   `variant` bits 0-3 pick the 64-bit Shoup-product code (0: compiler's
 *   64-bit products, 1: mad.wide high word, 2: carry-chain high word, 3:
 *   truncated high word from three partial products, lazy bound 4q, needs
 *   q < 2^61), bit 4 the inverse butterfly.  Returns butterflies per second.
 *   Synchronises `stream`.
 * hx_probe_copy_rate: copies `bytes` (a multiple of 16, both addresses
 *   16-byte aligned) from src to dst `iters` times with a grid of
 *   blocks_per_sm 256-thread blocks per SM doing 16-byte loads and stores;
 *   either side may be device memory or pinned host memory (reached through
 *   unified addressing over the CPU-GPU link).  Returns bytes per second
 *   (one copy's bytes, not read + write) and the per-copy time in *ms.
 * Errors: HX_ERR_NULL, HX_ERR_ARG, HX_ERR_NOMEM, HX_ERR_CUDA.
 */
uint64_t hx_launch_count(void);

/* Per-launch timing (instrumentation; off by default).
 *
 * hx_timing_enable(1, capacity): every NTT pass kernel and fused tensor pass
 *   that the library launches from now on records a CUDA event before and
 *   after itself on its own stream, for up to `capacity` launches (1 ..
 *   2^20; further launches are not recorded).  The events are created here,
 *   so recording allocates nothing.  hx_timing_enable(0, 0) stops recording;
 *   what was recorded stays until read.  Errors: HX_ERR_ARG, HX_ERR_CUDA.
 * hx_timing_read: waits for the recorded launches to finish, writes up to
 *   `cap` of them in launch order to h_out (kernel id and duration in ms),
 *   sets *n_out to the number written and clears the record (all of it,
 *   even beyond `cap`).  Must not run while another thread is launching
 *   library kernels that it wants recorded.  Errors: HX_ERR_NULL, HX_ERR_CUDA
 *   (an event failed; the others are still written).
 * hx_kernel_name: the kernel's name with its template arguments, as CUDA
 *   tools print it (e.g. "ntt_pass_kernel<1, 0, 3, 8, 1, 0>"), into buf.
 *   Errors: HX_ERR_NULL, HX_ERR_ARG (unknown id), HX_ERR_CAPACITY (len too
 *   small). */
typedef struct hx_launch_time {
    uint32_t kernel;   /* kernel id, for hx_kernel_name */
    uint32_t reserved;
    float ms;          /* launch duration between its two events */
    float reserved2;
} hx_launch_time;

int hx_timing_enable(int on, uint32_t capacity);
int hx_timing_read(hx_launch_time* h_out, uint32_t cap, uint32_t* n_out);
int hx_kernel_name(uint32_t kernel, char* buf, uint32_t len);
int hx_probe_int_mul_rate(uint32_t kind, uint32_t iters, double* ops_per_s, float* ms,
                          hx_stream_t stream);
int hx_probe_butterfly_rate(uint32_t variant, uint32_t iters, uint64_t q,
                            double* butterflies_per_s, float* ms, hx_stream_t stream);
int hx_probe_copy_rate(void* dst, const void* src, uint64_t bytes, uint32_t iters,
                       uint32_t blocks_per_sm, double* bytes_per_s, float* ms,
                       hx_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* HEXGPU_H */
