// Instantiations of the fused tensor / first-inverse-pass kernels with one
// output per block, and the menu of both kinds.
#include "ntt_tensor.cuh"

namespace hx {

TensorPassKernel pick_tensor_inv3(int K, bool tws);   // ntt_tensor3.cu

// Three outputs per block exist for 8 elements per thread (register budget).
TensorPassKernel pick_tensor_inv(int logR, int K, bool tws, int npf) {
    if (npf == 3) return logR == 3 ? pick_tensor_inv3(K, tws) : nullptr;
    if (logR == 3) return tws ? tensor_k<3, true, 1>(K) : tensor_k<3, false, 1>(K);
    if (logR == 4) return tws ? tensor_k<4, true, 1>(K) : tensor_k<4, false, 1>(K);
    return nullptr;
}

}  // namespace hx
