// Element-wise modular kernels (Section 3 free-function API, Section 3.3).
//
//   add / sub : (a +- b) mod q, inputs in [0, q)                  EltwiseAddMod
//   negate    : (q - a) mod q, input in [0, q)       element-wise negation
//   mult      : (a * b) mod q by Barrett with Q = bitlen(q),
//               L = 63 + Q, k = floor(2^L / q)  (Algorithm
//               "VectorVectorModMulAVX512Int"; inputs first reduced from
//               [0, k q) by conditional subtractions)             EltwiseMultMod
//   fma       : (a * s + d) mod q with the scalar's Shoup factor
//               s' = floor(s 2^64 / q) (Algorithm "EltwiseFMAModAVX512")
//   tensor    : d0 = A0 B0, d1 = A0 B1 + A1 B0, d2 = A1 B1, then
//               r_k = d_k s + e_k -- the element-wise middle of a
//               ciphertext product, fused so each operand is read once.
//
// These are HBM-bound (8 B per operand element, a few integer multiplies),
// so the kernels are plain grid-stride loops over 16-byte vectors, one
// modulus per block row, sized to fill all SMs.
#include <stdint.h>

#include <algorithm>

#include "hx_internal.h"
#include "modarith.cuh"

typedef unsigned __int128 u128;

namespace hx {

constexpr int kMaxLimbsPerLaunch = 64;

struct EltConsts {
    uint64_t q[kMaxLimbsPerLaunch];
    uint64_t bk[kMaxLimbsPerLaunch];   // Barrett k
    uint64_t s[kMaxLimbsPerLaunch];    // FMA scalar
    uint64_t sp[kMaxLimbsPerLaunch];   // its Shoup factor
    uint32_t qm1[kMaxLimbsPerLaunch];  // bitlen(q) - 1
};

struct EltGeom {
    uint64_t n;          // row length
    uint32_t n_limbs;    // limbs per polynomial (row stride between polys)
    uint32_t limb0;      // first limb of this launch
    uint32_t chunk;      // limbs in this launch
};

__device__ __forceinline__ uint64_t row_offset(const EltGeom& g, uint32_t row, uint32_t& li) {
    const uint32_t poly = row / g.chunk;
    li = row % g.chunk;
    return ((uint64_t)poly * g.n_limbs + g.limb0 + li) * g.n;
}

template <int OP, int INMF, bool ADDEND>
__device__ __forceinline__ uint64_t elt_apply(uint64_t a, uint64_t b, const EltConsts& c,
                                              uint32_t li) {
    const uint64_t q = c.q[li];
    if (OP == ELT_ADD) {
        uint64_t r = a + b;
        return r >= q ? r - q : r;
    } else if (OP == ELT_SUB) {
        return a >= b ? a - b : a + (q - b);
    } else if (OP == ELT_NEG) {
        return a == 0 ? 0 : q - a;
    } else if (OP == ELT_MULT) {
        a = small_mod<INMF>(a, q);
        b = small_mod<INMF>(b, q);
        Barrett br{q, c.bk[li], c.qm1[li]};
        return barrett_mulmod(a, b, br);
    } else {
        a = small_mod<INMF>(a, q);
        uint64_t r = fma_shoup(a, c.s[li], c.sp[li], q);
        if (ADDEND) {
            r += small_mod<INMF>(b, q);
            r = r >= q ? r - q : r;
        }
        return r;
    }
}

// 32 registers: with 256-thread blocks eight fit on an SM, so the grid of
// about eight blocks an SM (elt_grid) is resident in one wave.
template <int OP, int INMF, bool ADDEND>
__global__ void __maxnreg__(32) eltwise_kernel(uint64_t* __restrict__ r,
                                                      const uint64_t* __restrict__ a,
                                                      const uint64_t* __restrict__ b,
                                                      EltConsts c, EltGeom g) {
    uint32_t li;
    const uint64_t off = row_offset(g, blockIdx.y, li);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if ((g.n & 1) == 0) {
        const uint64_t nv = g.n >> 1;
        const ulonglong2* A = reinterpret_cast<const ulonglong2*>(a + off);
        const ulonglong2* B = reinterpret_cast<const ulonglong2*>(b ? b + off : nullptr);
        ulonglong2* Rv = reinterpret_cast<ulonglong2*>(r + off);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
            const ulonglong2 x = A[i];
            const ulonglong2 y = B ? B[i] : make_ulonglong2(0, 0);
            Rv[i] = make_ulonglong2(elt_apply<OP, INMF, ADDEND>(x.x, y.x, c, li),
                                    elt_apply<OP, INMF, ADDEND>(x.y, y.y, c, li));
        }
    } else {
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
            const uint64_t y = b ? b[off + i] : 0;
            r[off + i] = elt_apply<OP, INMF, ADDEND>(a[off + i], y, c, li);
        }
    }
}

template <int INMF>
__global__ void __launch_bounds__(256) tensor_fma_kernel(
    uint64_t* __restrict__ r0, uint64_t* __restrict__ r1, uint64_t* __restrict__ r2,
    const uint64_t* __restrict__ A0, const uint64_t* __restrict__ A1,
    const uint64_t* __restrict__ B0, const uint64_t* __restrict__ B1,
    const uint64_t* __restrict__ e0, const uint64_t* __restrict__ e1,
    const uint64_t* __restrict__ e2, EltConsts c, EltGeom g) {
    uint32_t li;
    const uint64_t off = row_offset(g, blockIdx.y, li);
    const uint64_t q = c.q[li];
    const Barrett br{q, c.bk[li], c.qm1[li]};
    const uint64_t s = c.s[li], sp = c.sp[li];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
        const uint64_t j = off + i;
        const uint64_t a0 = small_mod<INMF>(A0[j], q), a1 = small_mod<INMF>(A1[j], q);
        const uint64_t b0 = small_mod<INMF>(B0[j], q), b1 = small_mod<INMF>(B1[j], q);
        r0[j] = tensor_r(tensor_d(0, a0, a1, b0, b1, br), e0[j], s, sp, q);
        r1[j] = tensor_r(tensor_d(1, a0, a1, b0, b1, br), e1[j], s, sp, q);
        r2[j] = tensor_r(tensor_d(2, a0, a1, b0, b1, br), e2[j], s, sp, q);
    }
}

static void fill_consts(EltConsts& c, const uint64_t* h_moduli, const uint64_t* h_scalars,
                        uint32_t limb0, uint32_t chunk) {
    for (uint32_t i = 0; i < chunk; ++i) {
        const uint64_t q = h_moduli[limb0 + i];
        int Q = 0;
        while (Q < 64 && (q >> Q)) ++Q;  // bit length
        c.q[i] = q;
        c.qm1[i] = (uint32_t)(Q - 1);
        c.bk[i] = (uint64_t)(((u128)1 << (63 + Q)) / q);
        const uint64_t s = h_scalars ? h_scalars[limb0 + i] : 0;
        c.s[i] = s;
        c.sp[i] = (uint64_t)(((u128)s << 64) / q);
    }
}

static dim3 elt_grid(uint64_t n, uint32_t rows, int threads, bool vec) {
    static int sm_count = 0;
    if (!sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (!sm_count) sm_count = 152;
    }
    const uint64_t work = vec ? (n + 1) / 2 : n;
    uint64_t bx = (work + threads - 1) / threads;
    // about 8 resident blocks per SM in total across rows
    const uint64_t target = std::max<uint64_t>(1, (uint64_t)sm_count * 8 / std::max<uint32_t>(rows, 1));
    bx = std::max<uint64_t>(1, std::min(bx, std::max<uint64_t>(target, 1)));
    return dim3((unsigned)std::min<uint64_t>(bx, 1u << 20), rows);
}

template <int OP, int INMF, bool ADDEND>
static cudaError_t launch_one(uint64_t* r, const uint64_t* a, const uint64_t* b,
                              const EltConsts& c, const EltGeom& g, uint32_t n_polys,
                              cudaStream_t st) {
    const uint32_t rows_total = n_polys * g.chunk;
    for (uint32_t r0 = 0; r0 < rows_total; r0 += 65535u / g.chunk * g.chunk) {
        const uint32_t rows = std::min(rows_total - r0, 65535u / g.chunk * g.chunk);
        EltGeom gg = g;
        // offset whole polynomials
        const uint64_t poly_off = (uint64_t)(r0 / g.chunk) * g.n_limbs * g.n;
        dim3 grid = elt_grid(g.n, rows, 256, (g.n & 1) == 0);
        eltwise_kernel<OP, INMF, ADDEND><<<grid, 256, 0, st>>>(
            r + poly_off, a + poly_off, b ? b + poly_off : nullptr, c, gg);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int OP, bool ADDEND>
static cudaError_t dispatch_mf(uint32_t in_mf, uint64_t* r, const uint64_t* a, const uint64_t* b,
                               const EltConsts& c, const EltGeom& g, uint32_t n_polys,
                               cudaStream_t st) {
    switch (in_mf) {
        case 1: return launch_one<OP, 1, ADDEND>(r, a, b, c, g, n_polys, st);
        case 2: return launch_one<OP, 2, ADDEND>(r, a, b, c, g, n_polys, st);
        case 4: return launch_one<OP, 4, ADDEND>(r, a, b, c, g, n_polys, st);
        case 8: return launch_one<OP, 8, ADDEND>(r, a, b, c, g, n_polys, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_eltwise(int op, uint64_t* r, const uint64_t* a, const uint64_t* b,
                           const uint64_t* h_scalars, uint64_t n, const uint64_t* h_moduli,
                           uint32_t n_limbs, uint32_t n_polys, uint32_t in_mf,
                           cudaStream_t stream) {
    for (uint32_t limb0 = 0; limb0 < n_limbs; limb0 += kMaxLimbsPerLaunch) {
        const uint32_t chunk = std::min<uint32_t>(kMaxLimbsPerLaunch, n_limbs - limb0);
        EltConsts c;
        fill_consts(c, h_moduli, h_scalars, limb0, chunk);
        EltGeom g{n, n_limbs, limb0, chunk};
        cudaError_t e;
        switch (op) {
            case ELT_ADD: e = launch_one<ELT_ADD, 1, false>(r, a, b, c, g, n_polys, stream); break;
            case ELT_SUB: e = launch_one<ELT_SUB, 1, false>(r, a, b, c, g, n_polys, stream); break;
            case ELT_NEG: e = launch_one<ELT_NEG, 1, false>(r, a, b, c, g, n_polys, stream); break;
            case ELT_MULT: e = dispatch_mf<ELT_MULT, false>(in_mf, r, a, b, c, g, n_polys, stream); break;
            case ELT_FMA:
                e = b ? dispatch_mf<ELT_FMA, true>(in_mf, r, a, b, c, g, n_polys, stream)
                      : dispatch_mf<ELT_FMA, false>(in_mf, r, a, b, c, g, n_polys, stream);
                break;
            default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_tensor_fma(uint64_t* r0, uint64_t* r1, uint64_t* r2, const uint64_t* A0,
                              const uint64_t* A1, const uint64_t* B0, const uint64_t* B1,
                              const uint64_t* h_scalars, const uint64_t* e0, const uint64_t* e1,
                              const uint64_t* e2, uint64_t n, const uint64_t* h_moduli,
                              uint32_t n_limbs, uint32_t n_polys, uint32_t in_mf,
                              cudaStream_t stream) {
    for (uint32_t limb0 = 0; limb0 < n_limbs; limb0 += kMaxLimbsPerLaunch) {
        const uint32_t chunk = std::min<uint32_t>(kMaxLimbsPerLaunch, n_limbs - limb0);
        EltConsts c;
        fill_consts(c, h_moduli, h_scalars, limb0, chunk);
        EltGeom g{n, n_limbs, limb0, chunk};
        const uint32_t rows_total = n_polys * chunk;
        const uint32_t rows_max = 65535u / chunk * chunk;
        for (uint32_t rr = 0; rr < rows_total; rr += rows_max) {
            const uint32_t rows = std::min(rows_total - rr, rows_max);
            const uint64_t po = (uint64_t)(rr / chunk) * n_limbs * n;
            dim3 grid = elt_grid(n, rows, 256, false);
            switch (in_mf) {
                case 1:
                    tensor_fma_kernel<1><<<grid, 256, 0, stream>>>(r0 + po, r1 + po, r2 + po, A0 + po,
                        A1 + po, B0 + po, B1 + po, e0 + po, e1 + po, e2 + po, c, g);
                    break;
                case 2:
                    tensor_fma_kernel<2><<<grid, 256, 0, stream>>>(r0 + po, r1 + po, r2 + po, A0 + po,
                        A1 + po, B0 + po, B1 + po, e0 + po, e1 + po, e2 + po, c, g);
                    break;
                case 4:
                    tensor_fma_kernel<4><<<grid, 256, 0, stream>>>(r0 + po, r1 + po, r2 + po, A0 + po,
                        A1 + po, B0 + po, B1 + po, e0 + po, e1 + po, e2 + po, c, g);
                    break;
                default: return cudaErrorInvalidValue;
            }
            count_launch();
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace hx
