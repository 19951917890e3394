// Instantiations of the product-fused inverse first pass with the tile's
// twiddles staged in shared memory (menu in ntt_mul.cuh).
#include "ntt_mul.cuh"

namespace hx {

MulPassKernel pick_mul_inv_tws(int logR, int K, int np) { return mul_menu<true>(logR, K, np); }

}  // namespace hx
