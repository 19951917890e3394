// Instantiations of the fused tensor / first-inverse-pass kernels that
// compute and transform all three outputs of a ciphertext in one block.
#include "ntt_tensor.cuh"

namespace hx {

TensorPassKernel pick_tensor_inv3(int K, bool tws) {
    return tws ? tensor_k<3, true, 3>(K) : tensor_k<3, false, 3>(K);
}

}  // namespace hx
