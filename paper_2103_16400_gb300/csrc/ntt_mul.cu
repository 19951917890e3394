// Instantiations of the product-fused inverse first pass, twiddles through
// the read-only cache (menu in ntt_mul.cuh).
#include "ntt_mul.cuh"

namespace hx {

MulPassKernel pick_mul_inv(int logR, int K, int np, bool tws) {
    return tws ? pick_mul_inv_tws(logR, K, np) : mul_menu<false>(logR, K, np);
}

}  // namespace hx
