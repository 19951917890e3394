// Instantiations of the cluster-fused inverse transform with the ciphertext
// tensor computed in its first phase (ntt_cluster.cuh).
#include "ntt_cluster.cuh"

namespace hx {

ClusterTensorKernel pick_cluster_t(int logR, int K1, int K2) {
#define HX_ENTRY(a, b)                                                \
    if (K1 == a && K2 == b)                                           \
        return logR == 4 ? ntt_cluster_tensor_kernel<4, a, b>         \
                         : logR == 3 ? ntt_cluster_tensor_kernel<3, a, b> : nullptr;
    HX_CLUSTER_MENU(HX_ENTRY)
#undef HX_ENTRY
    return nullptr;
}

}  // namespace hx
