// FP64 form of the hydro kernels (every step in double precision).
#include "hydro.cuh"

namespace amm {
AMM_INSTANTIATE(double)
}
