// FP32 forms of the hydro kernels: float bulk arithmetic; double for the
// per-cell flux accumulation, the Newton guard and the conservation sums.
#include "hydro.cuh"
#include "individual.cuh"

namespace amm {
AMM_INSTANTIATE(float)
AMM_INSTANTIATE_INDIVIDUAL(float)
}
