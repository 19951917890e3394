// Instantiations of the inverse (Gentleman-Sande / Harvey) pass kernels with 2
// polynomial(s) per thread.
#include "ntt_inst.cuh"

namespace hx {

PassKernel pick_plain_i2(bool column, int logR, int K) {
    return menu<false, 2, 0>(column, logR, K);
}

}  // namespace hx
