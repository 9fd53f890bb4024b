// One persistent launch per step: every phase of the update (gradients +
// limiter, with the per-box Courant minimum on a moving mesh; on a static
// mesh the Courant minimum first and the predicted records with the
// gradients; face fluxes; cell update + conservation sums; per-box totals)
// runs in a single cooperative kernel whose CTAs walk the work items of each
// phase and meet at a grid barrier between phases.
// The batched ensemble (many independent boxes of uneven size, each with its
// own Courant step) is advanced with one such launch per step, replayed from
// a CUDA graph.
//
// The grid barrier is a counter and a generation word in global memory.  All
// CTAs are co-resident (cooperative launch, grid sized from the occupancy),
// and every wait is bounded: after BARRIER_POLLS polls the CTA records a
// timeout in the status word and continues, so the kernel always ends.
#include <cuda_runtime.h>

#pragma once

#include "hydro.cuh"

namespace amm {

constexpr unsigned BARRIER_POLLS = 1u << 22;

__device__ __forceinline__ void grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks,
                                             unsigned* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    if (arrived == nblocks - 1u) {
      *count = 0u;
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
    } else {
      unsigned polls = 0;
      while (*gen == g) {
        if (++polls > BARRIER_POLLS) {
          atomicOr(status, (unsigned)ST_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// three CTAs per SM: every phase runs at the occupancy of the heaviest one,
// and the two the register cap gives (90 registers) starve the latency-bound
// gradient and update phases (measured 0.33 -> 0.27 ms per 64^3 step)
template <typename real, int GG, bool ENT>
__global__ void __launch_bounds__(CELL_TILE, 3) k_step_persistent(HydroView<real> v, unsigned* bar) {
  if (v.pred) {
    // static mesh: the step before the gradients (v.pred is the same for all CTAs)
    for (int wi = blockIdx.x; wi < v.n_ctiles; wi += gridDim.x) courant_item<real>(v, wi);
    grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  }
  const int n_grad = v.n_ctiles * GG;
  for (int wi = blockIdx.x; wi < n_grad; wi += gridDim.x) grad_item<real, GG, ENT>(v, wi);
  grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  for (int wi = blockIdx.x; wi < v.n_ftiles; wi += gridDim.x) flux_item<real, FACE_TILE, ENT>(v, wi);
  grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  for (int wi = blockIdx.x; wi < v.n_ctiles; wi += gridDim.x) update_item<real, 1, ENT>(v, wi);
  grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  for (int b = blockIdx.x; b < v.nboxes; b += gridDim.x) finish_item<real, CELL_TILE>(v, b, 1);
}

template <typename real>
cudaError_t launch_step_persistent(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  v.update_lanes = 1;
  cudaError_t e = cudaMemsetAsync(c->cour_bits, 0xff, sizeof(unsigned long long) * c->nboxes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->fmax_bits, 0, sizeof(unsigned) * FMAX_STRIDE * c->nboxes, c->stream);
  if (e != cudaSuccess) return e;
  auto kern = c->opt.entropy ? k_step_persistent<real, 4, true> : k_step_persistent<real, 4, false>;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CELL_TILE, 0)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(per_sm * sms));
  cfg.blockDim = dim3(CELL_TILE);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, v, c->barrier);
}

}  // namespace amm
