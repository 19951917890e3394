// extern "C" entry points of libhexgpu: argument validation, then dispatch to
// the kernels.  Declarations and their documentation are in include/hexgpu.h.
#include <string.h>

#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "hx_internal.h"

using namespace hx;

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// [a, a + bytes) and [b, b + bytes) overlap without being the same range
bool partial_overlap(const void* a, const void* b, uint64_t bytes) {
    if (!a || !b || a == b) return false;
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return HX_OK;
    if (e == cudaErrorMemoryAllocation) return HX_ERR_NOMEM;
    return HX_ERR_CUDA;
}

int check_ntt(hx_plan_t plan, const uint64_t* r, const uint64_t* x, uint32_t n_polys,
              uint32_t in_mf, uint32_t out_mf, bool fwd) {
    if (!plan || !r || !x) return HX_ERR_NULL;
    if (!aligned16(r) || !aligned16(x)) return HX_ERR_ALIGN;
    if (n_polys == 0 || (uint64_t)n_polys * plan->n_limbs > (1ull << 31) / 1) return HX_ERR_ARG;
    if (fwd) {
        if (!(in_mf == 1 || in_mf == 2 || in_mf == 4)) return HX_ERR_MOD_FACTOR;
        if (!(out_mf == 1 || out_mf == 4)) return HX_ERR_MOD_FACTOR;
    } else {
        if (!(in_mf == 1 || in_mf == 2)) return HX_ERR_MOD_FACTOR;
        if (!(out_mf == 1 || out_mf == 2)) return HX_ERR_MOD_FACTOR;
    }
    const uint64_t bytes = (uint64_t)n_polys * plan->n_limbs * plan->N * 8;
    if (partial_overlap(r, x, bytes)) return HX_ERR_OVERLAP;
    return HX_OK;
}

int check_elt(const uint64_t* r, const uint64_t* a, const uint64_t* b, bool b_required, uint64_t n,
              const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys) {
    if (!r || !a || !h_moduli || (b_required && !b)) return HX_ERR_NULL;
    if (!aligned16(r) || !aligned16(a) || (b && !aligned16(b))) return HX_ERR_ALIGN;
    if (n == 0 || n_limbs == 0 || n_polys == 0) return HX_ERR_ARG;
    const uint64_t bytes = n * n_limbs * n_polys * 8;
    if (partial_overlap(r, a, bytes) || partial_overlap(r, b, bytes)) return HX_ERR_OVERLAP;
    return HX_OK;
}

struct RawKey {
    int device;
    uint64_t N;
    std::vector<uint64_t> moduli;
    bool operator<(const RawKey& o) const {
        return std::tie(device, N, moduli) < std::tie(o.device, o.N, o.moduli);
    }
};

std::mutex g_raw_mu;
std::map<RawKey, hx_plan_t>* g_raw_plans = nullptr;

int raw_plan(uint64_t N, const uint64_t* h_moduli, uint32_t n_limbs, hx_plan_t* out) {
    if (!h_moduli) return HX_ERR_NULL;
    if (n_limbs == 0) return HX_ERR_ARG;
    int dev = 0;
    cudaGetDevice(&dev);
    RawKey key{dev, N, std::vector<uint64_t>(h_moduli, h_moduli + n_limbs)};
    std::lock_guard<std::mutex> g(g_raw_mu);
    if (!g_raw_plans) g_raw_plans = new std::map<RawKey, hx_plan_t>();
    auto it = g_raw_plans->find(key);
    if (it != g_raw_plans->end()) {
        *out = it->second;
        return HX_OK;
    }
    hx_plan_t p = nullptr;
    int st = hx_plan_create(&p, N, h_moduli, n_limbs, nullptr);
    if (st != HX_OK) return st;
    (*g_raw_plans)[key] = p;
    *out = p;
    return HX_OK;
}

}  // namespace

extern "C" {

const char* hx_strerror(int s) {
    switch (s) {
        case HX_OK: return "success";
        case HX_ERR_NULL: return "a required pointer is NULL";
        case HX_ERR_ALIGN: return "a device pointer is not 16-byte aligned";
        case HX_ERR_DEGREE: return "N is not a power of two in [2^10, 2^17]";
        case HX_ERR_MODULUS: return "modulus not prime, not 1 mod 2N, or out of range";
        case HX_ERR_ROOT: return "supplied root is not a primitive 2N-th root of unity";
        case HX_ERR_MOD_FACTOR: return "input/output mod factor not allowed";
        case HX_ERR_CUDA: return "CUDA runtime error";
        case HX_ERR_ARG: return "argument out of range";
        case HX_ERR_OVERLAP: return "result and operand partially overlap";
        case HX_ERR_TIMEOUT: return "device-side wait timed out";
        case HX_ERR_NOMEM: return "allocation failed";
        case HX_ERR_CAPACITY: return "request exceeds the fixed scratch capacity";
        default: return "unknown status";
    }
}

int hx_abi_version(void) { return 1; }

int hx_ntt_forward(hx_plan_t plan, uint64_t* r, const uint64_t* x, uint32_t n_polys,
                   uint32_t in_mf, uint32_t out_mf, hx_stream_t stream) {
    int st = check_ntt(plan, r, x, n_polys, in_mf, out_mf, true);
    if (st != HX_OK) return st;
    return cuda_status(launch_ntt(plan, r, x, n_polys, true, in_mf, out_mf, plan->cfg_fwd,
                                  (cudaStream_t)stream));
}

int hx_ntt_inverse(hx_plan_t plan, uint64_t* r, const uint64_t* x, uint32_t n_polys,
                   uint32_t in_mf, uint32_t out_mf, hx_stream_t stream) {
    int st = check_ntt(plan, r, x, n_polys, in_mf, out_mf, false);
    if (st != HX_OK) return st;
    return cuda_status(launch_ntt(plan, r, x, n_polys, false, in_mf, out_mf, plan->cfg_inv,
                                  (cudaStream_t)stream));
}

int hx_ntt_forward_raw(uint64_t* d_ptr, uint64_t N, const uint64_t* h_moduli, uint32_t n_limbs,
                       uint32_t in_mf, uint32_t out_mf, hx_stream_t stream) {
    hx_plan_t p = nullptr;
    int st = raw_plan(N, h_moduli, n_limbs, &p);
    if (st != HX_OK) return st;
    return hx_ntt_forward(p, d_ptr, d_ptr, 1, in_mf, out_mf, stream);
}

int hx_ntt_inverse_raw(uint64_t* d_ptr, uint64_t N, const uint64_t* h_moduli, uint32_t n_limbs,
                       uint32_t in_mf, uint32_t out_mf, hx_stream_t stream) {
    hx_plan_t p = nullptr;
    int st = raw_plan(N, h_moduli, n_limbs, &p);
    if (st != HX_OK) return st;
    return hx_ntt_inverse(p, d_ptr, d_ptr, 1, in_mf, out_mf, stream);
}

static int check_moduli(const uint64_t* h_moduli, uint32_t n_limbs, uint64_t qmax, uint64_t qmin) {
    for (uint32_t l = 0; l < n_limbs; ++l)
        if (h_moduli[l] < qmin || h_moduli[l] > qmax) return HX_ERR_MODULUS;
    return HX_OK;
}

int hx_eltwise_add_mod(uint64_t* r, const uint64_t* a, const uint64_t* b, uint64_t n,
                       const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys,
                       hx_stream_t stream) {
    int st = check_elt(r, a, b, true, n, h_moduli, n_limbs, n_polys);
    if (st != HX_OK) return st;
    if ((st = check_moduli(h_moduli, n_limbs, (1ull << 63) - 1, 2)) != HX_OK) return st;
    return cuda_status(launch_eltwise(ELT_ADD, r, a, b, nullptr, n, h_moduli, n_limbs, n_polys, 1,
                                      (cudaStream_t)stream));
}

int hx_eltwise_sub_mod(uint64_t* r, const uint64_t* a, const uint64_t* b, uint64_t n,
                       const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys,
                       hx_stream_t stream) {
    int st = check_elt(r, a, b, true, n, h_moduli, n_limbs, n_polys);
    if (st != HX_OK) return st;
    if ((st = check_moduli(h_moduli, n_limbs, (1ull << 63) - 1, 2)) != HX_OK) return st;
    return cuda_status(launch_eltwise(ELT_SUB, r, a, b, nullptr, n, h_moduli, n_limbs, n_polys, 1,
                                      (cudaStream_t)stream));
}

int hx_eltwise_negate_mod(uint64_t* r, const uint64_t* a, uint64_t n, const uint64_t* h_moduli,
                          uint32_t n_limbs, uint32_t n_polys, hx_stream_t stream) {
    int st = check_elt(r, a, nullptr, false, n, h_moduli, n_limbs, n_polys);
    if (st != HX_OK) return st;
    if ((st = check_moduli(h_moduli, n_limbs, (1ull << 63) - 1, 2)) != HX_OK) return st;
    return cuda_status(launch_eltwise(ELT_NEG, r, a, nullptr, nullptr, n, h_moduli, n_limbs,
                                      n_polys, 1, (cudaStream_t)stream));
}

int hx_eltwise_mult_mod(uint64_t* r, const uint64_t* a, const uint64_t* b, uint64_t n,
                        const uint64_t* h_moduli, uint32_t n_limbs, uint32_t n_polys,
                        uint32_t in_mf, hx_stream_t stream) {
    int st = check_elt(r, a, b, true, n, h_moduli, n_limbs, n_polys);
    if (st != HX_OK) return st;
    if (!(in_mf == 1 || in_mf == 2 || in_mf == 4)) return HX_ERR_MOD_FACTOR;
    if ((st = check_moduli(h_moduli, n_limbs, (1ull << 62) - 1, 3)) != HX_OK) return st;
    for (uint32_t l = 0; l < n_limbs; ++l) {
        const uint64_t q = h_moduli[l];
        if ((q & (q - 1)) == 0) return HX_ERR_MODULUS;        // Barrett k needs q > 2^(Q-1)
        if ((unsigned __int128)in_mf * q >= ((unsigned __int128)1 << 63)) return HX_ERR_MOD_FACTOR;
    }
    return cuda_status(launch_eltwise(ELT_MULT, r, a, b, nullptr, n, h_moduli, n_limbs, n_polys,
                                      in_mf, (cudaStream_t)stream));
}

int hx_eltwise_fma_mod(uint64_t* r, const uint64_t* a, const uint64_t* h_scalars,
                       const uint64_t* d_addend, uint64_t n, const uint64_t* h_moduli,
                       uint32_t n_limbs, uint32_t n_polys, uint32_t in_mf, hx_stream_t stream) {
    if (!h_scalars) return HX_ERR_NULL;
    int st = check_elt(r, a, d_addend, false, n, h_moduli, n_limbs, n_polys);
    if (st != HX_OK) return st;
    if (!(in_mf == 1 || in_mf == 2 || in_mf == 4 || in_mf == 8)) return HX_ERR_MOD_FACTOR;
    if ((st = check_moduli(h_moduli, n_limbs, (1ull << 61) - 1, 2)) != HX_OK) return st;
    for (uint32_t l = 0; l < n_limbs; ++l)
        if (h_scalars[l] >= h_moduli[l]) return HX_ERR_ARG;
    return cuda_status(launch_eltwise(ELT_FMA, r, a, d_addend, h_scalars, n, h_moduli, n_limbs,
                                      n_polys, in_mf, (cudaStream_t)stream));
}

int hx_dyadic_tensor_fma(uint64_t* r0, uint64_t* r1, uint64_t* r2, const uint64_t* A0,
                         const uint64_t* A1, const uint64_t* B0, const uint64_t* B1,
                         const uint64_t* h_scalars, const uint64_t* e0, const uint64_t* e1,
                         const uint64_t* e2, uint64_t n, const uint64_t* h_moduli,
                         uint32_t n_limbs, uint32_t n_polys, uint32_t in_mf, hx_stream_t stream) {
    if (!r0 || !r1 || !r2 || !A0 || !A1 || !B0 || !B1 || !h_scalars || !e0 || !e1 || !e2 ||
        !h_moduli)
        return HX_ERR_NULL;
    if (n == 0 || n_limbs == 0 || n_polys == 0) return HX_ERR_ARG;
    if (!(in_mf == 1 || in_mf == 2 || in_mf == 4)) return HX_ERR_MOD_FACTOR;
    int st = check_moduli(h_moduli, n_limbs, (1ull << 61) - 1, 3);
    if (st != HX_OK) return st;
    for (uint32_t l = 0; l < n_limbs; ++l) {
        const uint64_t q = h_moduli[l];
        if ((q & (q - 1)) == 0) return HX_ERR_MODULUS;
        if (h_scalars[l] >= q) return HX_ERR_ARG;
    }
    const uint64_t bytes = n * n_limbs * n_polys * 8;
    const uint64_t* ins[7] = {A0, A1, B0, B1, e0, e1, e2};
    uint64_t* outs[3] = {r0, r1, r2};
    for (auto o : outs) {
        if (!aligned16(o)) return HX_ERR_ALIGN;
        for (auto i : ins) {
            // outputs may not alias inputs at all: each output element is
            // written after reading several inputs at the same index
            const uintptr_t x = (uintptr_t)o, y = (uintptr_t)i;
            if (x < y + bytes && y < x + bytes) return HX_ERR_OVERLAP;
        }
    }
    for (auto i : ins)
        if (!aligned16(i)) return HX_ERR_ALIGN;
    return cuda_status(launch_tensor_fma(r0, r1, r2, A0, A1, B0, B1, h_scalars, e0, e1, e2, n,
                                         h_moduli, n_limbs, n_polys, in_mf, (cudaStream_t)stream));
}

int hx_poly_mul(hx_plan_t plan, uint64_t* r, uint64_t* a, uint64_t* b, uint32_t n_polys,
                hx_stream_t stream) {
    if (!plan || !r || !a || !b) return HX_ERR_NULL;
    const uint64_t bytes = (uint64_t)n_polys * plan->n_limbs * plan->N * 8;
    if (a == b || partial_overlap(a, b, bytes)) return HX_ERR_OVERLAP;
    if (r != a && r != b && (partial_overlap(r, a, bytes) || partial_overlap(r, b, bytes)))
        return HX_ERR_OVERLAP;
    int st = hx_ntt_forward(plan, a, a, n_polys, 1, 4, stream);
    if (st != HX_OK) return st;
    if ((st = hx_ntt_forward(plan, b, b, n_polys, 1, 4, stream)) != HX_OK) return st;
    // the product computed in the inverse's first pass when its schedule
    // allows (a per-tile row pass), else a separate element-wise pass
    if (mul_fusable(plan->cfg_inv))
        return cuda_status(launch_mul_inverse(plan, r, a, b, n_polys, 4, plan->cfg_inv,
                                              (cudaStream_t)stream));
    st = cuda_status(launch_eltwise(ELT_MULT, r, a, b, nullptr, plan->N, plan->moduli.data(),
                                    plan->n_limbs, n_polys, 4, (cudaStream_t)stream));
    if (st != HX_OK) return st;
    return hx_ntt_inverse(plan, r, r, n_polys, 1, 1, stream);
}

int hx_dyadic_inverse(hx_plan_t plan, uint64_t* r, const uint64_t* A, const uint64_t* B,
                      uint32_t n_polys, uint32_t in_mf, hx_stream_t stream) {
    if (!plan || !r || !A || !B) return HX_ERR_NULL;
    if (!aligned16(r) || !aligned16(A) || !aligned16(B)) return HX_ERR_ALIGN;
    if (n_polys == 0 || (uint64_t)n_polys * plan->n_limbs > (1ull << 31)) return HX_ERR_ARG;
    if (!(in_mf == 1 || in_mf == 2 || in_mf == 4)) return HX_ERR_MOD_FACTOR;
    const uint64_t bytes = (uint64_t)n_polys * plan->n_limbs * plan->N * 8;
    // the result may be one of the spectra, or disjoint from both
    if ((r != A && partial_overlap(r, A, bytes)) || (r != B && partial_overlap(r, B, bytes)))
        return HX_ERR_OVERLAP;
    cudaStream_t s = (cudaStream_t)stream;
    if (mul_fusable(plan->cfg_inv))
        return cuda_status(launch_mul_inverse(plan, r, A, B, n_polys, in_mf, plan->cfg_inv, s));
    int st = cuda_status(launch_eltwise(ELT_MULT, r, A, B, nullptr, plan->N, plan->moduli.data(),
                                        plan->n_limbs, n_polys, in_mf, s));
    if (st != HX_OK) return st;
    return hx_ntt_inverse(plan, r, r, n_polys, 1, 1, stream);
}

int hx_tensor_fma_inverse(hx_plan_t plan, uint64_t* o0, uint64_t* o1, uint64_t* o2,
                          const uint64_t* A0, const uint64_t* A1, const uint64_t* B0,
                          const uint64_t* B1, const uint64_t* h_scalars, const uint64_t* e0,
                          const uint64_t* e1, const uint64_t* e2, uint32_t n_polys,
                          uint32_t in_mf, hx_stream_t stream) {
    if (!plan || !o0 || !o1 || !o2 || !A0 || !A1 || !B0 || !B1 || !h_scalars || !e0 || !e1 ||
        !e2)
        return HX_ERR_NULL;
    if (n_polys == 0 || (uint64_t)n_polys * 4 * plan->n_limbs > (1ull << 31)) return HX_ERR_ARG;
    const uint64_t S = (uint64_t)n_polys * plan->n_limbs * plan->N;
    const bool fused_layout = A1 == A0 + S && B0 == A0 + 2 * S && B1 == A0 + 3 * S &&
                              e1 == e0 + S && e2 == e0 + 2 * S && o1 == o0 + S && o2 == o0 + 2 * S;
    if (fused_layout && tensor_fusable(plan->cfg_inv)) {
        // the element-wise step's checks: moduli < 2^61, scalars < q,
        // alignment, outputs disjoint from every input
        if (!(in_mf == 1 || in_mf == 2 || in_mf == 4)) return HX_ERR_MOD_FACTOR;
        for (uint32_t l = 0; l < plan->n_limbs; ++l) {
            const uint64_t q = plan->moduli[l];
            if (q >= (1ull << 61)) return HX_ERR_MODULUS;
            if (h_scalars[l] >= q) return HX_ERR_ARG;
        }
        if (!aligned16(o0) || !aligned16(A0) || !aligned16(e0)) return HX_ERR_ALIGN;
        const uintptr_t x = (uintptr_t)o0, xe = x + 3 * S * 8;
        const uintptr_t a = (uintptr_t)A0, ae = a + 4 * S * 8;
        const uintptr_t e = (uintptr_t)e0, ee = e + 3 * S * 8;
        if ((x < ae && a < xe) || (x < ee && e < xe)) return HX_ERR_OVERLAP;
        return cuda_status(launch_tensor_inverse(plan, o0, A0, e0, n_polys, h_scalars, in_mf,
                                                 plan->cfg_inv, (cudaStream_t)stream));
    }
    int st = hx_dyadic_tensor_fma(o0, o1, o2, A0, A1, B0, B1, h_scalars, e0, e1, e2, plan->N,
                                  plan->moduli.data(), plan->n_limbs, n_polys, in_mf, stream);
    if (st != HX_OK) return st;
    if (o1 == o0 + S && o2 == o0 + 2 * S)
        return hx_ntt_inverse(plan, o0, o0, 3 * n_polys, 1, 1, stream);
    uint64_t* outs[3] = {o0, o1, o2};
    for (auto y : outs)
        if ((st = hx_ntt_inverse(plan, y, y, n_polys, 1, 1, stream)) != HX_OK) return st;
    return HX_OK;
}

int hx_poly_product(hx_plan_t plan, uint64_t* r, const uint64_t* a, const uint64_t* b,
                    uint64_t* work, uint32_t n_polys, hx_stream_t stream) {
    if (!plan || !r || !a || !b || !work) return HX_ERR_NULL;
    if (n_polys == 0 || (uint64_t)n_polys * 2 * plan->n_limbs > (1ull << 31)) return HX_ERR_ARG;
    if (!aligned16(r) || !aligned16(a) || !aligned16(b) || !aligned16(work)) return HX_ERR_ALIGN;
    const uint64_t S = (uint64_t)n_polys * plan->n_limbs * plan->N;
    const uintptr_t w = (uintptr_t)work, we = w + 2 * S * 8;
    const uintptr_t spans[3][2] = {{(uintptr_t)r, (uintptr_t)r + S * 8},
                                   {(uintptr_t)a, (uintptr_t)a + S * 8},
                                   {(uintptr_t)b, (uintptr_t)b + S * 8}};
    for (const auto& x : spans)
        if (x[0] < we && w < x[1]) return HX_ERR_OVERLAP;
    for (int k = 1; k < 3; ++k)   // the result: equal to an operand or apart from it
        if (spans[0][0] != spans[k][0] && spans[0][0] < spans[k][1] && spans[k][0] < spans[0][1])
            return HX_ERR_OVERLAP;
    const cudaStream_t s = (cudaStream_t)stream;
    if (mul_step_fusable(plan->cfg_fwd, plan->cfg_inv))
        return cuda_status(
            launch_mul_step(plan, r, a, b, work, n_polys, plan->cfg_fwd, plan->cfg_inv, s));
    int st = hx_ntt_forward(plan, work, a, n_polys, 1, 4, stream);
    if (st == HX_OK) st = hx_ntt_forward(plan, work + S, b, n_polys, 1, 4, stream);
    if (st != HX_OK) return st;
    return hx_dyadic_inverse(plan, r, work, work + S, n_polys, 4, stream);
}

int hx_ciphertext_step(hx_plan_t plan, uint64_t* r, const uint64_t* in, uint64_t* work,
                       const uint64_t* h_scalars, const uint64_t* e, uint32_t n_ct,
                       hx_stream_t stream) {
    if (!plan || !r || !in || !work || !h_scalars || !e) return HX_ERR_NULL;
    if (n_ct == 0 || (uint64_t)n_ct * 4 * plan->n_limbs > (1ull << 31)) return HX_ERR_ARG;
    for (uint32_t l = 0; l < plan->n_limbs; ++l) {
        const uint64_t q = plan->moduli[l];
        if (q >= (1ull << 61)) return HX_ERR_MODULUS;
        if (h_scalars[l] >= q) return HX_ERR_ARG;
    }
    if (!aligned16(r) || !aligned16(in) || !aligned16(work) || !aligned16(e)) return HX_ERR_ALIGN;
    const uint64_t S = (uint64_t)n_ct * plan->n_limbs * plan->N;
    const uintptr_t x = (uintptr_t)r, xe = x + 3 * S * 8;
    const uintptr_t a = (uintptr_t)in, ae = a + 4 * S * 8;
    const uintptr_t w = (uintptr_t)work, we = w + 4 * S * 8;
    const uintptr_t ea = (uintptr_t)e, ee = ea + 3 * S * 8;
    if ((x < ae && a < xe) || (x < we && w < xe) || (x < ee && ea < xe) ||
        (w < ee && ea < we) || (w != a && w < ae && a < we))
        return HX_ERR_OVERLAP;
    const cudaStream_t s = (cudaStream_t)stream;
    if (ct_step_fusable(plan->cfg_fwd, plan->cfg_inv))
        return cuda_status(
            launch_ct_step(plan, r, in, work, e, n_ct, h_scalars, plan->cfg_fwd, plan->cfg_inv, s));
    int st = hx_ntt_forward(plan, work, in, 4 * n_ct, 1, 4, stream);
    if (st != HX_OK) return st;
    return hx_tensor_fma_inverse(plan, r, r + S, r + 2 * S, work, work + S, work + 2 * S,
                                 work + 3 * S, h_scalars, e, e + S, e + 2 * S, n_ct, 4, stream);
}

int hx_ciphertext_tensor(hx_plan_t plan, uint64_t* o0, uint64_t* o1, uint64_t* o2, uint64_t* a0,
                         uint64_t* a1, uint64_t* b0, uint64_t* b1, const uint64_t* h_scalars,
                         const uint64_t* e0, const uint64_t* e1, const uint64_t* e2,
                         uint32_t n_polys, hx_stream_t stream) {
    if (!plan || !o0 || !o1 || !o2 || !a0 || !a1 || !b0 || !b1) return HX_ERR_NULL;
    for (uint32_t l = 0; l < plan->n_limbs; ++l)
        if (plan->moduli[l] >= (1ull << 61)) return HX_ERR_MODULUS;
    int st;
    // operands laid out back to back ([4][n_polys][limbs][N], [3][...]) are
    // transformed by one call each, which fills the GPU better than four/three
    const uint64_t S = (uint64_t)n_polys * plan->n_limbs * plan->N;
    uint64_t* ins[4] = {a0, a1, b0, b1};
    if (a1 == a0 + S && b0 == a0 + 2 * S && b1 == a0 + 3 * S && (uint64_t)n_polys * 4 < (1u << 31)) {
        if ((st = hx_ntt_forward(plan, a0, a0, 4 * n_polys, 1, 4, stream)) != HX_OK) return st;
    } else {
        for (auto x : ins)
            if ((st = hx_ntt_forward(plan, x, x, n_polys, 1, 4, stream)) != HX_OK) return st;
    }
    return hx_tensor_fma_inverse(plan, o0, o1, o2, a0, a1, b0, b1, h_scalars, e0, e1, e2, n_polys,
                                 4, stream);
}

}  // extern "C"
