// Face fluxes of the FP32 learned form: the flux kernel with the proposal
// network fused in.  Each CTA of 128 threads walks 128-face tiles
// (persistently); per tile every thread extrapolates its face (face_prepare),
// writes the normalised features as row t of a BF16 operand, one thread
// issues the two tensor-core layers (tcgen05, FP32 accumulators in tensor
// memory, 64 columns reused by both layers), every thread reads its row back,
// forms p0 = pbar exp(y) and runs the exact Riemann solver from it
// (face_finish).  Newton still iterates to the same tolerance, so the result
// does not depend on the network beyond the iteration count.
#include <cuda_runtime.h>

#include "hydro.cuh"
#include "learned.cuh"
#include "tc.cuh"

namespace amm {

constexpr int LT = 128;  // faces per tile = threads per CTA = MMA rows

struct LearnedSmem {
  alignas(1024) uint8_t a1[LT * 16 * 2];
  alignas(1024) uint8_t a2[LT * MLP_HID * 2];
  alignas(1024) uint8_t b1[MLP_HID * 16 * 2];
  alignas(1024) uint8_t b2[MLP_HID * MLP_HID * 2];
  float bias1[MLP_HID], bias2[MLP_HID], w3[MLP_HID], bias3;
  float hdt;
  uint64_t mbar;
  uint32_t tmem;
  uint32_t ok;
};

// SiLU from one hardware tanh: z sigma(z) = z/2 (1 + tanh(z/2)); the
// proposal only seeds Newton, so the approximate tanh is accurate enough
__device__ __forceinline__ float silu_fast(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return 0.5f * z * (1.0f + t);
}

__global__ void __launch_bounds__(LT, 4) k_flux_learned(HydroView<float> v, int nsub) {
  extern __shared__ uint8_t smem_raw[];
  LearnedSmem& s =
      *reinterpret_cast<LearnedSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const MlpDevice* M = (const MlpDevice*)v.mlp;
  const int t = threadIdx.x;
  const int warp = t >> 5;
  if (t < 32) tc::tmem_alloc(&s.tmem, 64);
  if (t == 0) {
    tc::mbar_init(&s.mbar, 1);
    s.ok = 1;
  }
  for (int i = t; i < MLP_HID * 16; i += LT)
    *reinterpret_cast<__nv_bfloat16*>(s.b1 + tc::kmajor_offset(i / 16, i % 16, 16)) = M->W1[i];
  for (int i = t; i < MLP_HID * MLP_HID; i += LT)
    *reinterpret_cast<__nv_bfloat16*>(s.b2 + tc::kmajor_offset(i / MLP_HID, i % MLP_HID, MLP_HID)) = M->W2[i];
  if (t < MLP_HID) {
    s.bias1[t] = M->b1[t];
    s.bias2[t] = M->b2[t];
    s.w3[t] = __bfloat162float(M->W3[t]);
  }
  if (t == 0) s.bias3 = M->b3;
  const uint32_t idesc = tc::make_idesc(128, 64);
  const float g = v.gas.g;
  uint32_t phase = 0;
  for (int st = blockIdx.x; st < nsub; st += gridDim.x) {
    const Tile tile = v.ftiles[st >> 1];
    const int first = tile.begin + (st & 1) * LT;
    const int k0 = first + t;
    const bool valid = k0 < tile.end;
    if (t == 0) s.hdt = (float)(0.5 * box_dt(v, tile.box));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    FaceWork<float> f;
    face_prepare(v, valid ? k0 : tile.begin, valid, s.hdt, f);
    // normalised features (the network's input)
    const float rb = 0.5f * (f.WppL[0] + f.WppR[0]);
    const float pb = 0.5f * (f.WppL[4] + f.WppR[4]);
    const float icb = rsqrtf(g * pb / rb);
    {
      const float irb = 1.0f / rb, ipb = 1.0f / pb;
      float row[16] = {__logf(f.WppL[0] * irb), __logf(f.WppL[4] * ipb), f.uL * icb, __logf(f.WppR[0] * irb),
                       __logf(f.WppR[4] * ipb), f.uR * icb, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      tc::st_bf16x8(s.a1, tc::kmajor_offset(t, 0, 16), row);
      tc::st_bf16x8(s.a1, tc::kmajor_offset(t, 8, 16), row + 8);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      tc::mma_bf16(s.tmem, tc::kmajor_desc(tc::smem_addr(s.a1), 16), tc::kmajor_desc(tc::smem_addr(s.b1), 16), idesc,
                   false);
      tc::mma_commit(&s.mbar);
    }
    if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
    phase ^= 1u;
    tc::fence_after_sync();
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float z[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, 16 * c), z);
#pragma unroll
      for (int j = 0; j < 16; j++) z[j] = silu_fast(z[j] + s.bias1[16 * c + j]);
      tc::st_bf16x8(s.a2, tc::kmajor_offset(t, 16 * c, MLP_HID), z);
      tc::st_bf16x8(s.a2, tc::kmajor_offset(t, 16 * c + 8, MLP_HID), z + 8);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
#pragma unroll
      for (int kb = 0; kb < MLP_HID / 16; kb++)
        tc::mma_bf16(s.tmem, tc::kmajor_desc(tc::smem_addr(s.a2) + 256 * kb, MLP_HID),
                     tc::kmajor_desc(tc::smem_addr(s.b2) + 256 * kb, MLP_HID), idesc, kb > 0);
      tc::mma_commit(&s.mbar);
    }
    if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
    phase ^= 1u;
    tc::fence_after_sync();
    float y = s.bias3;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float z[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, 16 * c), z);
#pragma unroll
      for (int j = 0; j < 16; j++) y += s.w3[16 * c + j] * silu_fast(z[j] + s.bias2[16 * c + j]);
    }
    y = fminf(fmaxf(y, -30.0f), 30.0f);
    const bool use = s.ok != 0;   // after a timed-out wait, fall back to the standard guess
    face_finish<float, LT>(v, f, tile.box, min(LT, tile.end - first), use, pb * __expf(y));
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t == 0 && !s.ok) atomicOr(&v.stats->status, (unsigned)ST_TIMEOUT);
  if (t < 32) tc::tmem_dealloc(s.tmem, 64);
}

static size_t learned_smem() { return sizeof(LearnedSmem) + 1024; }

cudaError_t prepare_flux_learned() {
  return cudaFuncSetAttribute(k_flux_learned, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)learned_smem());
}

cudaError_t launch_flux_learned(amm_ctx* c, const HydroView<float>& v) {
  if (!c->mlp) return cudaErrorInvalidValue;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nsub = 2 * c->n_ftiles;
  const int grid = std::min(nsub, 4 * sms);
  k_flux_learned<<<grid, LT, learned_smem(), c->stream>>>(v, nsub);
  return cudaGetLastError();
}

}  // namespace amm
