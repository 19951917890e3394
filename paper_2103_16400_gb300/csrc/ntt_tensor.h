// Arguments of the inverse-transform pass that computes the ciphertext tensor
// in its prologue (ntt_tensor.cu).
#pragma once
#include <stdint.h>

namespace hx {

struct PassArgs;

constexpr int kTensorLimbs = 64;   // limbs per launch (scalars travel as kernel parameters)

struct TensorIn {
    const uint64_t* A;   // A0 | A1 | B0 | B1 back to back: [4][n_ct][n_limbs][N], < in_mf q
    const uint64_t* E;   // e0 | e1 | e2 back to back: [3][n_ct][n_limbs][N], < q
    uint32_t n_ct;       // ciphertext pairs
    uint32_t in_mf;      // 1, 2 or 4
    uint32_t limb0;      // this launch covers limbs limb0 .. limb0 + gridDim.y - 1
    uint32_t pad_;
    uint64_t s[kTensorLimbs];    // per limb of the launch: scalar s_l ...
    uint64_t sp[kTensorLimbs];   // ... and its Shoup factor floor(s_l 2^64 / q_l)
};

typedef void (*TensorPassKernel)(PassArgs, TensorIn);

// ntt_tensor.cu: the fused first inverse pass for (elements per thread,
// stages, staged twiddles, outputs per block: 1 or 3), nullptr if not in
// the menu
TensorPassKernel pick_tensor_inv(int logR, int K, bool tws, int npf);

// ntt_ctrow.cu: the tensor step with both row passes around it (the
// forward's row stages on the four operands, the tensor, the inverse's row
// stages on the three outputs), for (elements per thread, stages); nullptr if
// not in the menu (8 elements a thread, 6..9 stages)
TensorPassKernel pick_ct_row(int logR, int K);

}  // namespace hx
