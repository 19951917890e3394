// Instantiations of the inverse (Gentleman-Sande / Harvey) pass kernels: the plain
// per-tile kernels and the persistent double-buffered ones.
#include "ntt_kernels.cuh"

namespace hx {

template <template <bool, bool, int, int> class Ker, bool COLUMN, int LOG_R>
static PassKernel inst(int K) {
    switch (K) {
        case 6: return Ker<false, COLUMN, LOG_R, 6>::fn;
        case 7: return Ker<false, COLUMN, LOG_R, 7>::fn;
        case 8: return Ker<false, COLUMN, LOG_R, 8>::fn;
        case 9: return Ker<false, COLUMN, LOG_R, 9>::fn;
        default: break;
    }
    if (!COLUMN) {
        switch (K) {
            case 10: return Ker<false, false, LOG_R, 10>::fn;
            case 11: return Ker<false, false, LOG_R, 11>::fn;
            case 12: return Ker<false, false, LOG_R, 12>::fn;
            case 13: return Ker<false, false, LOG_R, 13>::fn;
            default: break;
        }
    }
    return nullptr;
}

template <bool F, bool C, int R, int K>
struct Plain {
    static constexpr PassKernel fn = ntt_pass_kernel<F, C, R, K>;
};
template <bool F, bool C, int R, int K>
struct Pipe {
    static constexpr PassKernel fn = ntt_pipe_kernel<F, C, R, K>;
};

template <template <bool, bool, int, int> class Ker>
static PassKernel pick(bool column, int logR, int K) {
    if (logR == 3) return column ? inst<Ker, true, 3>(K) : inst<Ker, false, 3>(K);
    if (logR == 4) return column ? inst<Ker, true, 4>(K) : inst<Ker, false, 4>(K);
    return nullptr;
}

PassKernel pick_inv(bool column, int logR, int K) { return pick<Plain>(column, logR, K); }
PassKernel pick_inv_pipe(bool column, int logR, int K) { return pick<Pipe>(column, logR, K); }

}  // namespace hx
