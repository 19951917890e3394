// Menu of the inverse's first (row or single) pass with the dyadic product of
// two forward outputs computed in its staging step (the product of Listing 4
// fused into the inverse transform): the same shapes as the inverse pass
// kernels -- 8 elements a thread with one or two polynomials, 16 with one.
// Instantiated in ntt_mul.cu (twiddles through the read-only cache) and
// ntt_muls.cu (twiddles staged in shared memory) so the halves compile in
// parallel.
#pragma once
#include "ntt_inst.cuh"

namespace hx {

template <int R, int NP, bool TWS>
static MulPassKernel mul_k(int K) {
    switch (K) {
        case 6: return ntt_mul_inv_kernel<R, 6, NP, TWS>;
        case 7: return ntt_mul_inv_kernel<R, 7, NP, TWS>;
        case 8: return ntt_mul_inv_kernel<R, 8, NP, TWS>;
        case 9: return ntt_mul_inv_kernel<R, 9, NP, TWS>;
        case 10: return ntt_mul_inv_kernel<R, 10, NP, TWS>;
        case 11: return ntt_mul_inv_kernel<R, 11, NP, TWS>;
        case 12: return ntt_mul_inv_kernel<R, 12, NP, TWS>;
        case 13: return ntt_mul_inv_kernel<R, 13, NP, TWS>;
        default: return nullptr;
    }
}

template <bool TWS>
static MulPassKernel mul_menu(int logR, int K, int np) {
    if (logR == 3 && np == 1) return mul_k<3, 1, TWS>(K);
    if (logR == 3 && np == 2) return mul_k<3, 2, TWS>(K);
    if (logR == 4 && np == 1) return mul_k<4, 1, TWS>(K);
    return nullptr;
}

}  // namespace hx
