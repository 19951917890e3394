// Kernel menus: which (direction, column/row, elements per thread, stages,
// polynomials per thread) pass kernels exist, and how the launcher picks one.
// Each ntt_*.cu translation unit instantiates one slice of the menu so the
// slices compile in parallel.
#pragma once
#include "ntt_kernels.cuh"

namespace hx {

// MODE: 0 one block per tile, twiddles read through the read-only cache;
// 1 persistent double-buffered kernel; 2 one block per tile with the tile's
// twiddles staged in shared memory.
template <bool F, int NP, int MODE, bool C, int R, int K>
static PassKernel menu_entry() {
    if constexpr (MODE == 1)
        return ntt_pipe_kernel<F, C, R, K>;
    else
        return ntt_pass_kernel<F, C, R, K, NP, MODE == 2>;
}

template <bool F, int NP, int MODE, bool C, int R>
static PassKernel menu_k(int K) {
    switch (K) {
        case 6: return menu_entry<F, NP, MODE, C, R, 6>();
        case 7: return menu_entry<F, NP, MODE, C, R, 7>();
        case 8: return menu_entry<F, NP, MODE, C, R, 8>();
        case 9: return menu_entry<F, NP, MODE, C, R, 9>();
        default: break;
    }
    if constexpr (!C) {   // single-pass and long row passes
        switch (K) {
            case 10: return menu_entry<F, NP, MODE, false, R, 10>();
            case 11: return menu_entry<F, NP, MODE, false, R, 11>();
            case 12: return menu_entry<F, NP, MODE, false, R, 12>();
            case 13: return menu_entry<F, NP, MODE, false, R, 13>();
            default: break;
        }
    }
    return nullptr;
}

// NP > 1 exists for 8 elements per thread only (register budget).
template <bool F, int NP, int MODE>
static PassKernel menu(bool column, int logR, int K) {
    if (logR == 3) return column ? menu_k<F, NP, MODE, true, 3>(K) : menu_k<F, NP, MODE, false, 3>(K);
    if constexpr (NP == 1) {
        if (logR == 4)
            return column ? menu_k<F, NP, MODE, true, 4>(K) : menu_k<F, NP, MODE, false, 4>(K);
    }
    return nullptr;
}

}  // namespace hx
