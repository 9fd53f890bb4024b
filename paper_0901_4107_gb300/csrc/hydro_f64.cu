// FP64 form of the hydro kernels (every step in double precision).
#include "hydro.cuh"
#include "individual.cuh"

namespace amm {
AMM_INSTANTIATE(double)
AMM_INSTANTIATE_INDIVIDUAL(double)

cudaError_t launch_individual_next(amm_ctx* c, const IndView& d) {
  k_ind_next<<<1, 32, 0, c->stream>>>(d);
  return cudaGetLastError();
}
}
