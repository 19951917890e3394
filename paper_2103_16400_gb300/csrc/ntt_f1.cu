// Instantiations of the forward (Cooley-Tukey / Harvey) pass kernels with 1
// polynomial(s) per thread, and of the persistent double-buffered ones.
#include "ntt_inst.cuh"

namespace hx {

PassKernel pick_plain_f1(bool column, int logR, int K) {
    return menu<true, 1, 0>(column, logR, K);
}

PassKernel pick_pipe_f(bool column, int logR, int K) {
    return menu<true, 1, 1>(column, logR, K);
}

}  // namespace hx
