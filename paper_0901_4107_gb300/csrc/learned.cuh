// Learned starting value for the Riemann star pressure (FP32 learned form).
//
// A 6 -> 64 -> 64 -> 1 multilayer perceptron with SiLU activations maps the
// normalised face state to a correction y of the two-shock estimate p_TS: the
// proposal log(p*/pbar) = log(p_TS/pbar) + y, i.e. Newton starts from
// p_TS exp(y).  The exact iteration still runs to the same tolerance, so the
// proposal changes the iteration count, not the answer.
// Features: with rhobar = (rho_L+rho_R)/2, pbar = (p_L+p_R)/2 and
// cbar = sqrt(gamma pbar / rhobar):
//   x = (log(rho_L/rhobar), log(p_L/pbar), u_L/cbar,
//        log(rho_R/rhobar), log(p_R/pbar), u_R/cbar).
// The paper has no counterpart; this is the specification of the learned form.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "amm.h"


namespace amm {

constexpr int MLP_IN = 6;
constexpr int MLP_HID = 64;

// The proposal stands in for the two-shock estimate only where the linearised
// estimate exceeds PROPOSAL_GATE times the larger side pressure (strong
// compression): for weaker compression the two-shock estimate is accurate to
// ~1e-4 or better, below what a BF16 network reaches, and replacing it costs
// Newton iterations.  A CTA whose faces all lie below the gate skips the
// network altogether.
constexpr float PROPOSAL_GATE = (float)AMM_PROPOSAL_GATE;

// Weights as the kernels consume them: BF16 matrices (row = output unit),
// FP32 biases.  W1 is padded to 16 inputs (zeros beyond 6).
struct MlpDevice {
  __nv_bfloat16 W1[MLP_HID * 16];
  __nv_bfloat16 W2[MLP_HID * MLP_HID];
  __nv_bfloat16 W3[MLP_HID];
  float b1[MLP_HID];
  float b2[MLP_HID];
  float b3;
};

}  // namespace amm
