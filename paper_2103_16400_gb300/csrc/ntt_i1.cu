// Instantiations of the inverse (Gentleman-Sande / Harvey) pass kernels with 1
// polynomial(s) per thread, and of the persistent double-buffered ones.
#include "ntt_inst.cuh"

namespace hx {

PassKernel pick_plain_i1(bool column, int logR, int K) {
    return menu<false, 1, 0>(column, logR, K);
}

PassKernel pick_pipe_i(bool column, int logR, int K) {
    return menu<false, 1, 1>(column, logR, K);
}

}  // namespace hx
