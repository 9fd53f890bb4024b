// Throughput probe of the FP32 and FP64 fused multiply-add pipes.  The flux
// kernels' ALU rooflines divide their counted FLOPs per second by this rate,
// measured on the same device in the same run (the clocks of the run apply).
//
// Each thread advances 8 independent chains x <- x * a + b, so one warp keeps
// the pipe's latency covered; 4 CTAs of 256 threads per SM.  The chains
// converge to b / (1 - a), so nothing overflows, and the final sums are
// compared (and stored to a device variable if the impossible happens) so
// the compiler keeps every chain.
#include <cuda_runtime.h>

#include "amm.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;
constexpr int PK_CTAS_PER_SM = 4;

static __device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_fma_chains(int iters, T a, T b) {
  T x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; c++) x[c] = (T)(threadIdx.x & 7) + (T)c;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; c++) x[c] = fma(x[c], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; c++) s += x[c];
  if (s == (T)-1) g_peak_sink = (double)s;   // never true (the chains stay positive); keeps them live
}

}  // namespace

extern "C" int amm_alu_peak(int fp64, int iters, double* flop_out, float* ms_out, void* stream) {
  if (iters < 1 || !flop_out || !ms_out) return AMM_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AMM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return AMM_ERR_CUDA;
  const cudaStream_t st = (cudaStream_t)stream;
  const int grid = sms * PK_CTAS_PER_SM;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return AMM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AMM_ERR_CUDA;
  }
  cudaEventRecord(e0, st);
  if (fp64)
    k_fma_chains<double><<<grid, PK_THREADS, 0, st>>>(iters, 0.999, 1e-3);
  else
    k_fma_chains<float><<<grid, PK_THREADS, 0, st>>>(iters, 0.999f, 1e-3f);
  cudaEventRecord(e1, st);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  const cudaError_t err2 = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || err2 != cudaSuccess || cudaGetLastError() != cudaSuccess) return AMM_ERR_CUDA;
  *flop_out = 2.0 * PK_CHAINS * (double)iters * (double)grid * PK_THREADS;
  *ms_out = ms;
  return AMM_OK;
}
