// The persistent single-launch step, FP32 forms (built with the same
// fast single-precision flags as the per-phase kernels of hydro_f32.cu, so
// both step modes give bit-identical results).
#include "persistent.cuh"

namespace amm {
template cudaError_t launch_step_persistent<float>(amm_ctx*, double);
}
