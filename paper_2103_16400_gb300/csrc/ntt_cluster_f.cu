// Instantiations of the cluster-fused forward transform (ntt_cluster.cuh).
#include "ntt_cluster.cuh"

namespace hx {

ClusterKernel pick_cluster_f(int logR, int K1, int K2) {
#define HX_ENTRY(a, b)                                                \
    if (K1 == a && K2 == b)                                           \
        return logR == 4 ? ntt_cluster_kernel<true, 4, a, b>          \
                         : logR == 3 ? ntt_cluster_kernel<true, 3, a, b> : nullptr;
    HX_CLUSTER_MENU(HX_ENTRY)
#undef HX_ENTRY
    return nullptr;
}

}  // namespace hx
