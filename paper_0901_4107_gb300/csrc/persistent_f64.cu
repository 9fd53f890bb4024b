// The persistent single-launch step, FP64 form.
#include "persistent.cuh"

namespace amm {
template cudaError_t launch_step_persistent<double>(amm_ctx*, double);
}
