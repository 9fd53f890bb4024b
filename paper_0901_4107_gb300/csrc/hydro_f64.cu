// FP64 form of the hydro kernels (every step in double precision).
#include "hydro.cuh"
#include "individual.cuh"

namespace amm {
AMM_INSTANTIATE(double)
AMM_INSTANTIATE_INDIVIDUAL(double)
}
