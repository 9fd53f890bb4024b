// amm_timestep_noalloc: the Courant time step for callers that cannot
// allocate device memory.
//
// Who needs it: code whose device memory is entirely owned by another
// allocator (a framework's caching pool that has reserved most of HBM, so a
// cudaMalloc here could fail), and code on a latency-critical path that must
// not call cudaMalloc/cudaFree because those calls can synchronise the whole
// device.  Such callers pass their own input and output buffers; the only
// working memory is the file-scope array below.
//
// The per-CTA partial minima live in g_courant_partials, a static __device__
// array of AMM_NOALLOC_MAX_BLOCKS doubles (128 KiB) that every GPU loading
// this library holds until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host it is only a stand-in symbol), so the
// device address is looked up with cudaGetSymbolAddress once per device, the
// first time this entry point runs on that device with it current; that first
// call should therefore happen before any stream capture.  All calls share the
// array: two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on it.  No slot needs clearing between calls:
// the first kernel writes every slot the second one reads.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "amm.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 16;
constexpr int NA_CELLS_PER_BLOCK = NA_THREADS * NA_CELLS_PER_THREAD;
constexpr int NA_MAX_BLOCKS = AMM_NOALLOC_MAX_BLOCKS;
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_courant_partials[NA_MAX_BLOCKS];

std::mutex g_mu;
double* g_partials_ptr[NA_MAX_DEVICES] = {nullptr};

// per-CTA minimum of R_i / (c_i + |v_i - w_i|) over its chunk of cells
__global__ void k_courant_partials(int64_t n, int dim, const double* W, const double* V, const double* wmesh,
                                   double gamma, double* partials) {
  const int nv = dim + 2;
  double m = INFINITY;
  const int64_t base = (int64_t)blockIdx.x * NA_CELLS_PER_BLOCK;
  for (int r = 0; r < NA_CELLS_PER_THREAD; r++) {
    const int64_t i = base + (int64_t)r * NA_THREADS + threadIdx.x;
    if (i >= n) break;
    const double* w = W + i * nv;
    const double rho = w[0], P = w[dim + 1];
    double vr = 0.0;
    for (int d = 0; d < dim; d++) {
      const double dv = w[1 + d] - (wmesh ? wmesh[i * dim + d] : 0.0);
      vr += dv * dv;
    }
    const double R = (dim == 3) ? cbrt(3.0 * V[i] / (4.0 * M_PI)) : sqrt(V[i] / M_PI);
    const double t = R / (sqrt(gamma * P / rho) + sqrt(vr));
    m = t < m ? t : m;   // a NaN cell never wins the minimum
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, m, o);
    m = u < m ? u : m;
  }
  __shared__ double wm[NA_THREADS / 32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = wm[0];
    for (int k = 1; k < NA_THREADS / 32; k++) b = wm[k] < b ? wm[k] : b;
    partials[blockIdx.x] = b;
  }
}

// dt = cfl * min over the partials
__global__ void k_courant_final(int nblocks, const double* partials, double cfl, double* dt_out) {
  double m = INFINITY;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) m = partials[k] < m ? partials[k] : m;
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, m, o);
    m = u < m ? u : m;
  }
  __shared__ double wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = wm[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) b = wm[k] < b ? wm[k] : b;
    *dt_out = cfl * b;
  }
}

}  // namespace

extern "C" int amm_timestep_noalloc(int dim, int64_t n_cells, const double* W_device, const double* V_device,
                                    const double* wmesh_device, double gamma, double cfl, double* dt_device,
                                    void* stream) {
  if ((dim != 2 && dim != 3) || n_cells < 1 || !W_device || !V_device || !dt_device) return AMM_ERR_INVALID_ARG;
  if (!(gamma > 1.0) || !(cfl > 0.0)) return AMM_ERR_INVALID_ARG;
  if (n_cells > AMM_NOALLOC_MAX_CELLS) return AMM_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return AMM_ERR_CUDA;
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_courant_partials);
      if (e != cudaSuccess || p == nullptr) return AMM_ERR_CUDA;
      g_partials_ptr[dev] = (double*)p;
    }
    partials = g_partials_ptr[dev];
  }
  const int nblocks = (int)((n_cells + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
  cudaStream_t st = (cudaStream_t)stream;
  k_courant_partials<<<nblocks, NA_THREADS, 0, st>>>(n_cells, dim, W_device, V_device, wmesh_device, gamma,
                                                     partials);
  if (cudaGetLastError() != cudaSuccess) return AMM_ERR_CUDA;
  k_courant_final<<<1, 1024, 0, st>>>(nblocks, partials, cfl, dt_device);
  if (cudaGetLastError() != cudaSuccess) return AMM_ERR_CUDA;
  return AMM_OK;
}
