// Internal declarations shared by the translation units of libhexgpu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <vector>

#include "hexgpu.h"   // include/ is on the include path

namespace hx {

// Per-limb constants resident on the device (one array per plan).
struct LimbDev {
    uint64_t q;
    uint64_t two_q;
    const ulonglong2* fwd;  // [N] {W, W'}: W = psi^brv(k), W' its Shoup factor
    const ulonglong2* inv;  // [N] {W, W'}: W = psi^-brv(k)
    uint64_t ninv, ninv_p;      // N^-1 and its Shoup factor
    uint64_t ninv_w, ninv_w_p;  // N^-1 * psi^-brv(1) and its Shoup factor
    uint32_t narrow;            // 1: q < 2^30, 32-bit words, beta = 2^32
    uint32_t barrett_qm1;       // bitlen(q) - 1 (Barrett shift)
    uint64_t barrett_k;         // floor(2^(63 + bitlen(q)) / q)
    uint32_t trunc;             // 1: 64-bit words with q < 2^61 -- the NTT uses the
                                // truncated-quotient Shoup product (values < 8q)
    uint32_t pad_;
};

// One pass of a transform: CT stages [s0, s0 + K) on tiles of
// 2^logGb (top-index values) x 2^K x 2^logGc (low-index values) elements,
// 2^logR elements per thread; pipe selects the persistent double-buffered
// kernel (1) or one block per tile (0); np = polynomials per thread sharing
// one set of twiddle registers (1 or 2; 2 only with logR 3 and pipe 0).
struct PassCfg {
    int s0, K, logGb, logGc, logR, pipe, np;
};

struct NttCfg {
    int npass;
    PassCfg pass[2];
};

// Device twiddle tables of one (device, N, q, psi): fwd[N] then inv[N] pairs,
// shared by every plan that uses them (plan.cpp keeps the cache).
struct TableEntry {
    int device = 0;
    void* d_mem = nullptr;
    size_t bytes = 0;
    LimbDev ld{};            // constants with fwd/inv pointing into d_mem
    ~TableEntry();
};

}  // namespace hx

struct hx_plan_s {
    uint64_t N = 0;
    int logN = 0;
    uint32_t n_limbs = 0;
    int device = 0;
    std::vector<uint64_t> moduli, roots;
    std::vector<std::shared_ptr<hx::TableEntry>> tables;   // one per limb (may repeat)
    hx::LimbDev* d_limbs = nullptr;
    std::vector<hx::LimbDev> h_limbs;
    // Launch order of the limbs in the fused tensor pass and the column
    // passes (fewer, longer blocks than the row passes): grid row y
    // transforms limb d_order[y].  Costliest limbs first (64-bit exact-quotient, then
    // truncated-quotient, then 32-bit words), stable, permuted within runs of
    // 64 limbs (the fused tensor pass launches at most 64 at a time), so that
    // the blocks that finish a pass are the short ones.  Device copy inside
    // the d_limbs allocation.
    uint32_t* d_order = nullptr;
    std::vector<uint32_t> h_order;
    uint64_t device_bytes = 0;
    bool cyclic = false;               // cyclic NTT over omega (else negacyclic over psi)
    hx::NttCfg cfg_fwd{}, cfg_inv{};   // kernel schedules per direction
};

namespace hx {

// probe.cu: counts kernel launches made by this library (all entry points)
void count_launch(uint64_t n = 1);
// probe.cu: per-launch timing (hx_timing_enable); timing_begin returns 0 when
// off or full, else a slot to pass to timing_end after the launch.  Kernel
// ids: bits 0-1 kind (0 per-tile pass, 1 persistent pass, 2 fused tensor
// pass, 3 cluster-fused transform), 2 forward, 3 column, 4-6 logR, 7-11 K
// (K1 for kind 3), 12-13 polynomials (outputs for the fused pass; for kind 3
// bit 12 marks the tensor-fused inverse) per block, 14 staged twiddles,
// 15-19 K2 (kind 3); for kind 0, bit 15 marks the inverse's first pass with
// the dyadic product fused in; for kind 2, bit 16 marks the step kernels that
// also run the forward's row stages (ntt_ctrow.cu), bit 17 the product's.
uint32_t timing_begin(cudaStream_t s, uint32_t kernel);
void timing_end(uint32_t slot, cudaStream_t s);

// plan.cpp
bool is_prime_u64(uint64_t n);
uint64_t powmod_u64(uint64_t a, uint64_t e, uint64_t q);
uint64_t min_primitive_root(uint64_t N, uint64_t q);
uint64_t min_primitive_nth_root(uint64_t N, uint64_t q);
std::vector<uint32_t> launch_order(const std::vector<LimbDev>& limbs);
NttCfg default_cfg(int logN, bool forward);
int acquire_tables(int device, uint64_t N, int logN, const std::vector<uint64_t>& moduli,
                   const std::vector<uint64_t>& roots, bool cyclic,
                   std::vector<std::shared_ptr<TableEntry>>* out);

// ntt.cu
cudaError_t launch_ntt(const hx_plan_s* plan, uint64_t* out, const uint64_t* in,
                       uint32_t n_polys, bool forward, uint32_t in_mf, uint32_t out_mf,
                       const NttCfg& cfg, cudaStream_t stream);
bool cfg_supported(int logN, const NttCfg& cfg);
// Inverse transform of the three ciphertext-tensor terms with the element-
// wise step in its first pass: out = [3][n_ct][limbs][N] from A = [4][n_ct]..
// (forward outputs, < in_mf q) and E = [3][n_ct].. (< q).  cudaErrorNotSupported
// when the schedule's first inverse pass is not a per-tile row pass.
bool tensor_fusable(const NttCfg& cfg);
// Inverse transform of the dyadic product a_i b_i mod q (a, b forward
// outputs below in_mf q) with the product computed in the inverse's first
// pass: out = InvNTT(a . b).  cudaErrorNotSupported when that pass is not a
// per-tile row pass (mul_fusable).
bool mul_fusable(const NttCfg& cfg);
cudaError_t launch_mul_inverse(const hx_plan_s* plan, uint64_t* out, const uint64_t* a,
                               const uint64_t* b, uint32_t n_polys, uint32_t in_mf,
                               const NttCfg& cfg, cudaStream_t stream);
cudaError_t launch_tensor_inverse(const hx_plan_s* plan, uint64_t* out, const uint64_t* A,
                                  const uint64_t* E, uint32_t n_ct, const uint64_t* h_scalars,
                                  uint32_t in_mf, const NttCfg& cfg, cudaStream_t stream);
// The whole ciphertext step in three launches: the forward's column pass
// (in -> work, the four operands back to back), the forward's row stages,
// the tensor and the inverse's row stages in one kernel (work, E -> out,
// ntt_ctrow.cu), the inverse's column pass (out, in place).  Needs both
// schedules two-pass with row passes over the same stages (ct_step_fusable;
// the inverse's row tile serves both), else cudaErrorNotSupported.
bool ct_step_fusable(const NttCfg& f, const NttCfg& i);
// The polynomial product in four launches: the forward's column pass of a
// and of b (into work = a | b), the forward's row stages, the dyadic product
// and the inverse's row stages in one kernel (work -> out, ntt_ctrow.cu), the
// inverse's column pass.  Needs both schedules two-pass over the same split
// (mul_step_fusable), else cudaErrorNotSupported.
bool mul_step_fusable(const NttCfg& f, const NttCfg& i);
cudaError_t launch_mul_step(const hx_plan_s* plan, uint64_t* out, const uint64_t* a,
                            const uint64_t* b, uint64_t* work, uint32_t n_polys,
                            const NttCfg& f, const NttCfg& i, cudaStream_t stream);
cudaError_t launch_ct_step(const hx_plan_s* plan, uint64_t* out, const uint64_t* in,
                           uint64_t* work, const uint64_t* E, uint32_t n_ct,
                           const uint64_t* h_scalars, const NttCfg& f, const NttCfg& i,
                           cudaStream_t stream);

// eltwise.cu
enum EltOp { ELT_ADD = 0, ELT_SUB = 1, ELT_MULT = 2, ELT_FMA = 3, ELT_NEG = 4 };
cudaError_t launch_eltwise(int op, uint64_t* r, const uint64_t* a, const uint64_t* b,
                           const uint64_t* h_scalars, uint64_t n, const uint64_t* h_moduli,
                           uint32_t n_limbs, uint32_t n_polys, uint32_t in_mf,
                           cudaStream_t stream);
cudaError_t launch_tensor_fma(uint64_t* r0, uint64_t* r1, uint64_t* r2, const uint64_t* A0,
                              const uint64_t* A1, const uint64_t* B0, const uint64_t* B1,
                              const uint64_t* h_scalars, const uint64_t* e0, const uint64_t* e1,
                              const uint64_t* e2, uint64_t n, const uint64_t* h_moduli,
                              uint32_t n_limbs, uint32_t n_polys, uint32_t in_mf,
                              cudaStream_t stream);

}  // namespace hx
