// Instantiations of the forward (Cooley-Tukey / Harvey) pass kernels with 2 polynomial(s) per
// thread and the tile's twiddles staged in shared memory.
#include "ntt_inst.cuh"

namespace hx {

PassKernel pick_tws_f2(bool column, int logR, int K) {
    return menu<true, 2, 2>(column, logR, K);
}

}  // namespace hx
