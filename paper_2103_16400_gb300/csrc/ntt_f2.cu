// Instantiations of the forward (Cooley-Tukey / Harvey) pass kernels with 2
// polynomial(s) per thread.
#include "ntt_inst.cuh"

namespace hx {

PassKernel pick_plain_f2(bool column, int logR, int K) {
    return menu<true, 2, 0>(column, logR, K);
}

}  // namespace hx
