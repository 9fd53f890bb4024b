// Learned starting value for the Riemann star pressure (FP32 learned form).
//
// A 6 -> 64 -> 64 -> 1 multilayer perceptron with SiLU activations maps the
// normalised face state to y = log(p* / pbar) and the Newton iteration
// starts from pbar exp(y); the exact iteration still runs to the same
// tolerance, so the proposal changes the iteration count, not the answer.
// Features: with rhobar = (rho_L+rho_R)/2, pbar = (p_L+p_R)/2 and
// cbar = sqrt(gamma pbar / rhobar):
//   x = (log(rho_L/rhobar), log(p_L/pbar), u_L/cbar,
//        log(rho_R/rhobar), log(p_R/pbar), u_R/cbar).
// The paper has no counterpart; this is the specification of the learned form.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "riemann.cuh"

namespace amm {

constexpr int MLP_IN = 6;
constexpr int MLP_HID = 64;

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

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

// Per-thread inference on the CUDA cores (reference form of the fused
// inference; the flux kernel of the learned form uses the tensor-core tile
// version in learned_tc.cuh).
template <typename real>
__device__ __forceinline__ real learned_guess(const void* mlp, real rhoL, real pL, real uL, real rhoR, real pR,
                                              real uR, const GasC<real>& G) {
  const MlpDevice* M = (const MlpDevice*)mlp;
  const float rb = 0.5f * ((float)rhoL + (float)rhoR);
  const float pb = 0.5f * ((float)pL + (float)pR);
  const float cb = sqrtf((float)G.g * pb / rb);
  const float x[6] = {__logf((float)rhoL / rb), __logf((float)pL / pb), (float)uL / cb,
                      __logf((float)rhoR / rb), __logf((float)pR / pb), (float)uR / cb};
  float h1[MLP_HID];
#pragma unroll 8
  for (int o = 0; o < MLP_HID; o++) {
    float z = M->b1[o];
#pragma unroll
    for (int k = 0; k < 6; k++) z += __bfloat162float(M->W1[o * 16 + k]) * x[k];
    h1[o] = silu_f(z);
  }
  float y = M->b3;
  for (int o = 0; o < MLP_HID; o++) {
    float z = M->b2[o];
#pragma unroll 16
    for (int k = 0; k < MLP_HID; k++) z += __bfloat162float(M->W2[o * MLP_HID + k]) * h1[k];
    y += __bfloat162float(M->W3[o]) * silu_f(z);
  }
  y = fminf(fmaxf(y, -40.0f), 40.0f);
  return (real)(pb * __expf(y));
}

}  // namespace amm
