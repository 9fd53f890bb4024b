// Learned starting value for the Riemann star pressure: the 6 -> 64 -> 64 -> 1
// SiLU perceptron on BF16 tensor cores (tcgen05, accumulators in tensor
// memory), its training (forward, backward, Adam), and the data path that
// feeds it (face-state harvest, exact p* targets, feature normalisation).
// The paper has no such component; see learned.cuh for the specification.
//
// Tiles are 128 samples (faces), one per thread of a 4-warp CTA, so sample t
// of the tile is row t of every MMA and lane t of tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "amm_internal.cuh"
#include "learned.cuh"
#include "riemann.cuh"
#include "tc.cuh"

namespace amm {

constexpr int MLP_TILE = 128;
constexpr int NP_W1 = MLP_HID * MLP_IN, NP_B1 = MLP_HID, NP_W2 = MLP_HID * MLP_HID, NP_B2 = MLP_HID, NP_W3 = MLP_HID;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NP_W1, OFF_W2 = OFF_B1 + NP_B1, OFF_B2 = OFF_W2 + NP_W2,
              OFF_W3 = OFF_B2 + NP_B2, OFF_B3 = OFF_W3 + NP_W3, NPARAMS = OFF_B3 + 1;

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// BF16 weights + FP32 biases from FP32 master parameters
__global__ void k_mlp_pack(const float* p, MlpDevice* out) {
  for (int i = threadIdx.x; i < MLP_HID * 16; i += blockDim.x) {
    const int o = i / 16, k = i % 16;
    out->W1[i] = __float2bfloat16_rn(k < MLP_IN ? p[OFF_W1 + o * MLP_IN + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < MLP_HID * MLP_HID; i += blockDim.x) out->W2[i] = __float2bfloat16_rn(p[OFF_W2 + i]);
  for (int i = threadIdx.x; i < MLP_HID; i += blockDim.x) {
    out->W3[i] = __float2bfloat16_rn(p[OFF_W3 + i]);
    out->b1[i] = p[OFF_B1 + i];
    out->b2[i] = p[OFF_B2 + i];
  }
  if (threadIdx.x == 0) out->b3 = p[OFF_B3];
}

// Shared-memory image of one CTA's operands
struct MlpSmem {
  alignas(1024) uint8_t a1[MLP_TILE * 16 * 2];        // X      [128 x 16]
  alignas(1024) uint8_t a2[MLP_TILE * MLP_HID * 2];   // H1     [128 x 64]
  alignas(1024) uint8_t b1[MLP_HID * 16 * 2];         // W1     [64 x 16]
  alignas(1024) uint8_t b2[MLP_HID * MLP_HID * 2];    // W2     [64 x 64]
  float bias1[MLP_HID], bias2[MLP_HID], w3[MLP_HID];
  float bias3;
  uint64_t mbar;
  uint32_t tmem;
  uint32_t ok;
};

// weights into the K-major core-matrix layout
__device__ __forceinline__ void load_weights(MlpSmem& s, const MlpDevice* M) {
  for (int i = threadIdx.x; i < MLP_HID * 16; i += blockDim.x) {
    const int o = i / 16, k = i % 16;
    *reinterpret_cast<__nv_bfloat16*>(s.b1 + tc::kmajor_offset(o, k, 16)) = M->W1[i];
  }
  for (int i = threadIdx.x; i < MLP_HID * MLP_HID; i += blockDim.x) {
    const int o = i / MLP_HID, k = i % MLP_HID;
    *reinterpret_cast<__nv_bfloat16*>(s.b2 + tc::kmajor_offset(o, k, MLP_HID)) = M->W2[i];
  }
  for (int i = threadIdx.x; i < MLP_HID; i += blockDim.x) {
    s.bias1[i] = M->b1[i];
    s.bias2[i] = M->b2[i];
    s.w3[i] = __bfloat162float(M->W3[i]);
  }
  if (threadIdx.x == 0) s.bias3 = M->b3;
}

// Forward pass of one tile; x[6] in, returns y.  Called by all 128 threads;
// uses tensor-memory columns [0,64) and [64,128) of s.tmem.  `phase` is the
// mbarrier parity of the first of the two waits (the second uses phase^1).
// On a wait timeout s.ok is cleared and y is 0.
__device__ __forceinline__ float mlp_tile_forward(MlpSmem& s, const float* x, uint32_t phase) {
  const int t = threadIdx.x;
  const int warp = t >> 5;
  {
    float row[16] = {x[0], x[1], x[2], x[3], x[4], x[5], 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    tc::st_bf16x8(s.a1, tc::kmajor_offset(t, 0, 16), row);
    tc::st_bf16x8(s.a1, tc::kmajor_offset(t, 8, 16), row + 8);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (t == 0) {
    const uint64_t ad = tc::kmajor_desc(tc::smem_addr(s.a1), 16);
    const uint64_t bd = tc::kmajor_desc(tc::smem_addr(s.b1), 16);
    tc::mma_bf16(s.tmem, ad, bd, tc::make_idesc(128, 64), false);
    tc::mma_commit(&s.mbar);
  }
  if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
  tc::fence_after_sync();
  // layer 1 epilogue: h1 = silu(z1 + b1) -> A2
#pragma unroll
  for (int c = 0; c < 4; c++) {
    float z[16];
    tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, 16 * c), z);
#pragma unroll
    for (int j = 0; j < 16; j++) z[j] = silu(z[j] + s.bias1[16 * c + j]);
    tc::st_bf16x8(s.a2, tc::kmajor_offset(t, 16 * c, MLP_HID), z);
    tc::st_bf16x8(s.a2, tc::kmajor_offset(t, 16 * c + 8, MLP_HID), z + 8);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (t == 0) {
#pragma unroll
    for (int kb = 0; kb < MLP_HID / 16; kb++) {
      const uint64_t ad = tc::kmajor_desc(tc::smem_addr(s.a2) + 256 * kb, MLP_HID);
      const uint64_t bd = tc::kmajor_desc(tc::smem_addr(s.b2) + 256 * kb, MLP_HID);
      tc::mma_bf16(s.tmem + 64, ad, bd, tc::make_idesc(128, 64), kb > 0);
    }
    tc::mma_commit(&s.mbar);
  }
  if (!tc::mbar_wait(&s.mbar, phase ^ 1u)) s.ok = 0;
  tc::fence_after_sync();
  float y = s.bias3;
#pragma unroll
  for (int c = 0; c < 4; c++) {
    float z[16];
    tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, 64 + 16 * c), z);
#pragma unroll
    for (int j = 0; j < 16; j++) y += s.w3[16 * c + j] * silu(z[j] + s.bias2[16 * c + j]);
  }
  return s.ok ? y : 0.0f;
}

// batched inference: one 128-sample tile per CTA
__global__ void __launch_bounds__(MLP_TILE) k_mlp_forward(const MlpDevice* M, const float* x, int64_t m, float* y,
                                                         unsigned* status) {
  extern __shared__ uint8_t smem_raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int t = threadIdx.x;
  if (t < 32) tc::tmem_alloc(&s.tmem, 128);
  if (t == 0) {
    tc::mbar_init(&s.mbar, 1);
    s.ok = 1;
  }
  load_weights(s, M);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const int64_t row = (int64_t)blockIdx.x * MLP_TILE + t;
  float xi[6] = {0, 0, 0, 0, 0, 0};
  if (row < m)
    for (int j = 0; j < 6; j++) xi[j] = x[row * 6 + j];
  const float yo = mlp_tile_forward(s, xi, 0);
  if (row < m) y[row] = yo;
  tc::fence_before_sync();
  __syncthreads();
  if (t == 0 && !s.ok) atomicOr(status, (unsigned)ST_TIMEOUT);
  if (t < 32) tc::tmem_dealloc(s.tmem, 128);
}


// ---------------------------------------------------------------- training
// Shared memory of the gradient kernel (one CTA per SM: it holds 512 TMEM
// columns).  Operands are K-major no-swizzle tiles (tc.cuh).
struct TrainSmem {
  alignas(1024) uint8_t a1[MLP_TILE * 16 * 2];        // X        [128 x 16]
  alignas(1024) uint8_t a2[MLP_TILE * MLP_HID * 2];   // H1       [128 x 64]
  alignas(1024) uint8_t a3[MLP_TILE * MLP_HID * 2];   // dZ2      [128 x 64]
  alignas(1024) uint8_t aw[128 * MLP_TILE * 2];       // [dZ2^T; dZ1^T]  [128 x 128 samples]
  alignas(1024) uint8_t bw[80 * MLP_TILE * 2];        // [H1^T; X^T]     [80 x 128 samples]
  alignas(1024) uint8_t b1[MLP_HID * 16 * 2];         // W1       [64 x 16]
  alignas(1024) uint8_t b2[MLP_HID * MLP_HID * 2];    // W2       [64 x 64]
  alignas(1024) uint8_t b2t[MLP_HID * MLP_HID * 2];   // W2^T     [64 x 64]
  float red[MLP_TILE][MLP_HID + 1];                   // per-sample rows for column sums
  float bias1[MLP_HID], bias2[MLP_HID], w3[MLP_HID], bias3;
  float acc_b1[MLP_HID], acc_b2[MLP_HID], acc_w3[MLP_HID], acc_b3, acc_loss;
  float lsum[MLP_TILE], dsum[MLP_TILE];
  uint64_t mbar;
  uint32_t tmem;
  uint32_t ok;
};

// TMEM columns: [0,64) Z1, [64,128) Z2, [128,192) dH1, [256,336) weight grads
constexpr int TC_Z1 = 0, TC_Z2 = 64, TC_DH1 = 128, TC_DW = 256;

__device__ __forceinline__ void tr_sync() {
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

// column sums of red[0..127][0..63] into acc (thread j < 64 owns column j;
// fixed row order)
__device__ __forceinline__ void tr_colsum(TrainSmem& s, float* acc) {
  __syncthreads();
  if (threadIdx.x < MLP_HID) {
    float a = 0.0f;
    for (int r = 0; r < MLP_TILE; r++) a += s.red[r][threadIdx.x];
    acc[threadIdx.x] += a;
  }
  __syncthreads();
}

// Gradient of L = sum over the batch of (y - t)^2 / n_total with respect to
// every parameter; each CTA processes tiles blockIdx.x, blockIdx.x+gridDim.x,
// ... of the batch and writes its partial sums to part[blockIdx.x][NPARAMS+1]
// (the last entry is its share of the loss).
__global__ void __launch_bounds__(MLP_TILE, 1) k_mlp_grads(const MlpDevice* M, const float* x, const float* tgt,
                                                          const int* idx, int64_t n, float inv_n, float* part,
                                                          unsigned* status) {
  extern __shared__ uint8_t smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int t = threadIdx.x;
  const int warp = t >> 5;
  if (t < 32) tc::tmem_alloc(&s.tmem, 512);
  if (t == 0) {
    tc::mbar_init(&s.mbar, 1);
    s.ok = 1;
    s.acc_b3 = 0.0f;
    s.acc_loss = 0.0f;
  }
  if (t < MLP_HID) s.acc_b1[t] = s.acc_b2[t] = s.acc_w3[t] = 0.0f;
  // weights: W1, W2 and W2^T in the operand layout
  for (int i = t; i < MLP_HID * 16; i += MLP_TILE)
    *reinterpret_cast<__nv_bfloat16*>(s.b1 + tc::kmajor_offset(i / 16, i % 16, 16)) = M->W1[i];
  for (int i = t; i < MLP_HID * MLP_HID; i += MLP_TILE) {
    const int o = i / MLP_HID, k = i % MLP_HID;
    *reinterpret_cast<__nv_bfloat16*>(s.b2 + tc::kmajor_offset(o, k, MLP_HID)) = M->W2[i];
    *reinterpret_cast<__nv_bfloat16*>(s.b2t + tc::kmajor_offset(k, o, MLP_HID)) = M->W2[i];
  }
  if (t < MLP_HID) {
    s.bias1[t] = M->b1[t];
    s.bias2[t] = M->b2[t];
    s.w3[t] = __bfloat162float(M->W3[t]);
  }
  if (t == 0) s.bias3 = M->b3;
  tr_sync();
  const uint32_t idesc64 = tc::make_idesc(128, 64), idesc80 = tc::make_idesc(128, 80);
  const int64_t tiles = (n + MLP_TILE - 1) / MLP_TILE;
  uint32_t phase = 0;
  bool first = true;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row = tile * MLP_TILE + t;
    const bool valid = row < n;
    const int64_t src = valid ? (idx ? (int64_t)idx[row] : row) : 0;
    float xi[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    float ti = 0.0f;
    if (valid) {
      for (int j = 0; j < MLP_IN; j++) xi[j] = x[src * MLP_IN + j];
      ti = tgt[src];
    }
    // X into A1 (row t) and into the rows 64.. of Bw (column t)
    tc::st_bf16x8(s.a1, tc::kmajor_offset(t, 0, 16), xi);
    tc::st_bf16x8(s.a1, tc::kmajor_offset(t, 8, 16), xi + 8);
#pragma unroll
    for (int j = 0; j < 16; j++)
      *reinterpret_cast<__nv_bfloat16*>(s.bw + tc::kmajor_offset(64 + j, t, MLP_TILE)) =
          __float2bfloat16_rn(valid ? xi[j] : 0.0f);
    tr_sync();
    if (t == 0) {
      tc::mma_bf16(s.tmem + TC_Z1, tc::kmajor_desc(tc::smem_addr(s.a1), 16), tc::kmajor_desc(tc::smem_addr(s.b1), 16),
                   idesc64, false);
      tc::mma_commit(&s.mbar);
    }
    if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
    phase ^= 1u;
    tc::fence_after_sync();
    // H1 = silu(Z1 + b1) -> A2 (row t) and Bw rows 0..63 (column t)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float z[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_Z1 + 16 * c), z);
#pragma unroll
      for (int j = 0; j < 16; j++) {
        z[j] = silu(z[j] + s.bias1[16 * c + j]);
        *reinterpret_cast<__nv_bfloat16*>(s.bw + tc::kmajor_offset(16 * c + j, t, MLP_TILE)) =
            __float2bfloat16_rn(valid ? z[j] : 0.0f);
      }
      tc::st_bf16x8(s.a2, tc::kmajor_offset(t, 16 * c, MLP_HID), z);
      tc::st_bf16x8(s.a2, tc::kmajor_offset(t, 16 * c + 8, MLP_HID), z + 8);
    }
    tr_sync();
    if (t == 0) {
#pragma unroll
      for (int kb = 0; kb < 4; kb++)
        tc::mma_bf16(s.tmem + TC_Z2, tc::kmajor_desc(tc::smem_addr(s.a2) + 256 * kb, MLP_HID),
                     tc::kmajor_desc(tc::smem_addr(s.b2) + 256 * kb, MLP_HID), idesc64, kb > 0);
      tc::mma_commit(&s.mbar);
    }
    if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
    phase ^= 1u;
    tc::fence_after_sync();
    // y, residual, dy = 2 (y - t) / n_total
    float y = s.bias3;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float z[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_Z2 + 16 * c), z);
#pragma unroll
      for (int j = 0; j < 16; j++) y += s.w3[16 * c + j] * silu(z[j] + s.bias2[16 * c + j]);
    }
    const float r = valid ? (y - ti) : 0.0f;
    const float dy = 2.0f * r * inv_n;
    s.lsum[t] = r * r * inv_n;
    s.dsum[t] = dy;
    // dW3 = sum dy h2 ; dZ2 = dy w3 silu'(Z2 + b2) -> A3 (row t), Aw rows 0..63 (column t)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float z[16], d[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_Z2 + 16 * c), z);
#pragma unroll
      for (int j = 0; j < 16; j++) {
        const float zz = z[j] + s.bias2[16 * c + j];
        s.red[t][16 * c + j] = dy * silu(zz);
        d[j] = dy * s.w3[16 * c + j] * dsilu(zz);
        *reinterpret_cast<__nv_bfloat16*>(s.aw + tc::kmajor_offset(16 * c + j, t, MLP_TILE)) =
            __float2bfloat16_rn(d[j]);
      }
      tc::st_bf16x8(s.a3, tc::kmajor_offset(t, 16 * c, MLP_HID), d);
      tc::st_bf16x8(s.a3, tc::kmajor_offset(t, 16 * c + 8, MLP_HID), d + 8);
    }
    tr_colsum(s, s.acc_w3);
    if (t == 0) {  // loss and db3 = sum dy, in sample order
      float l = 0.0f, b = 0.0f;
      for (int q = 0; q < MLP_TILE; q++) {
        l += s.lsum[q];
        b += s.dsum[q];
      }
      s.acc_loss += l;
      s.acc_b3 += b;
    }
    // db2 = sum dZ2 in FP32 (the BF16 copy in A3 is for the tensor core)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float z[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_Z2 + 16 * c), z);
#pragma unroll
      for (int j = 0; j < 16; j++) s.red[t][16 * c + j] = dy * s.w3[16 * c + j] * dsilu(z[j] + s.bias2[16 * c + j]);
    }
    tr_colsum(s, s.acc_b2);
    tr_sync();
    // dH1 = dZ2 W2
    if (t == 0) {
#pragma unroll
      for (int kb = 0; kb < 4; kb++)
        tc::mma_bf16(s.tmem + TC_DH1, tc::kmajor_desc(tc::smem_addr(s.a3) + 256 * kb, MLP_HID),
                     tc::kmajor_desc(tc::smem_addr(s.b2t) + 256 * kb, MLP_HID), idesc64, kb > 0);
      tc::mma_commit(&s.mbar);
    }
    if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
    phase ^= 1u;
    tc::fence_after_sync();
    // dZ1 = dH1 silu'(Z1 + b1) -> Aw rows 64..127 (column t); db1 = sum dZ1
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float z[16], h[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_Z1 + 16 * c), z);
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_DH1 + 16 * c), h);
#pragma unroll
      for (int j = 0; j < 16; j++) {
        const float d = valid ? h[j] * dsilu(z[j] + s.bias1[16 * c + j]) : 0.0f;
        s.red[t][16 * c + j] = d;
        *reinterpret_cast<__nv_bfloat16*>(s.aw + tc::kmajor_offset(64 + 16 * c + j, t, MLP_TILE)) =
            __float2bfloat16_rn(d);
      }
    }
    tr_colsum(s, s.acc_b1);
    tr_sync();
    // weight gradients: D[128 x 80] += Aw[128 x 128] Bw[80 x 128]^T
    if (t == 0) {
#pragma unroll
      for (int kb = 0; kb < MLP_TILE / 16; kb++)
        tc::mma_bf16(s.tmem + TC_DW, tc::kmajor_desc(tc::smem_addr(s.aw) + 256 * kb, MLP_TILE),
                     tc::kmajor_desc(tc::smem_addr(s.bw) + 256 * kb, MLP_TILE), idesc80, !(first && kb == 0));
      tc::mma_commit(&s.mbar);
    }
    if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
    phase ^= 1u;
    tc::fence_after_sync();
    first = false;
  }
  // partial gradients of this CTA
  float* out = part + (size_t)blockIdx.x * (NPARAMS + 1);
  if (!first) {
    // rows 0..63 x columns 0..63: dW2[o][i]; rows 64..127 x columns 64..69: dW1[i][j]
    if (warp < 2) {
#pragma unroll
      for (int c = 0; c < 4; c++) {
        float z[16];
        tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_DW + 16 * c), z);
#pragma unroll
        for (int j = 0; j < 16; j++) out[OFF_W2 + t * MLP_HID + 16 * c + j] = z[j];
      }
    } else {
      float z[16];
      tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, warp, TC_DW + 64), z);
#pragma unroll
      for (int j = 0; j < MLP_IN; j++) out[OFF_W1 + (t - 64) * MLP_IN + j] = z[j];
    }
  } else {
    for (int i = t; i < NP_W2; i += MLP_TILE) out[OFF_W2 + i] = 0.0f;
    for (int i = t; i < NP_W1; i += MLP_TILE) out[OFF_W1 + i] = 0.0f;
  }
  if (t < MLP_HID) {
    out[OFF_B1 + t] = s.acc_b1[t];
    out[OFF_B2 + t] = s.acc_b2[t];
    out[OFF_W3 + t] = s.acc_w3[t];
  }
  if (t == 0) {
    out[OFF_B3] = s.acc_b3;
    out[NPARAMS] = s.acc_loss;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t == 0 && !s.ok) atomicOr(status, (unsigned)ST_TIMEOUT);
  if (t < 32) tc::tmem_dealloc(s.tmem, 512);
}

// ordered sum of the per-CTA partials (bit reproducible)
__global__ void k_mlp_reduce(const float* part, int nparts, float* grads) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > NPARAMS) return;
  float a = 0.0f;
  for (int c = 0; c < nparts; c++) a += part[(size_t)c * (NPARAMS + 1) + i];
  grads[i] = a;
}

// Adam (Kingma & Ba) on the FP32 master parameters, then the BF16 repack
__global__ void k_mlp_adam(float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAMS) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// normalised features and pbar from face states (rhoL, uL, pL, rhoR, uR, pR)
__global__ void k_mlp_features(double gamma, int64_t m, const float* st, float* x, float* pbar, float* pts,
                               float* ratio) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float* s = st + 6 * i;
  if (pts || ratio) {
    // the two-shock estimate the proposal corrects, and the compression
    // measure of the gate, in FP32 as the flux kernel takes them
    const GasC<float> G(gamma);
    const float cL = sqrtf(G.g * s[2] / s[0]), cR = sqrtf(G.g * s[5] / s[3]);
    const float ppv = linearised_pstar(s[0], s[1], s[2], cL, s[3], s[4], s[5], cR);
    if (pts) pts[i] = two_shock_pstar(s[0], s[1], s[2], s[3], s[4], s[5], ppv, G);
    if (ratio) ratio[i] = ppv / fmaxf(s[2], s[5]);
  }
  const float rb = 0.5f * (s[0] + s[3]);
  const float pb = 0.5f * (s[2] + s[5]);
  const float cb = sqrtf((float)gamma * pb / rb);
  float* o = x + 6 * i;
  o[0] = logf(s[0] / rb);
  o[1] = logf(s[2] / pb);
  o[2] = s[1] / cb;
  o[3] = logf(s[3] / rb);
  o[4] = logf(s[5] / pb);
  o[5] = s[4] / cb;
  if (pbar) pbar[i] = pb;
}

// exact star pressure in FP64 (Newton from the standard guess to tol); NaN
// where the states generate vacuum (no star region)
__global__ void k_riemann_pstar(double gamma, int64_t m, const float* st, double tol, int maxit, float* pstar) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float* s = st + 6 * i;
  const double rL = s[0], uL = s[1], pL = s[2], rR = s[3], uR = s[4], pR = s[5];
  const GasC<double> G(gamma);
  const double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  if (!(rL > 0.0) || !(rR > 0.0) || !(pL > 0.0) || !(pR > 0.0) || G.two_gm1 * (cL + cR) <= uR - uL) {
    pstar[i] = __int_as_float(0x7fc00000);
    return;
  }
  RiemannInfo info{0, 0, 0, 0};
  NewtonTail<double> nt;
  const double p0 = standard_guess(rL, uL, pL, cL, rR, uR, pR, cR, G);
  const double p = newton_pstar(p0, rL, uL, pL, cL, rR, uR, pR, cR, G, tol, tol, maxit, info, nt);
  pstar[i] = info.fail ? __int_as_float(0x7fc00000) : (float)p;
}

// training target of each face state: log(p* / p_TS), the correction of the
// two-shock estimate (FP32, as the flux kernel forms it) that takes it to the
// exact star pressure (FP64 Newton to tol); NaN without a star region
__global__ void k_mlp_targets(double gamma, int64_t m, const float* st, double tol, int maxit, float* target) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float* s = st + 6 * i;
  const double rL = s[0], uL = s[1], pL = s[2], rR = s[3], uR = s[4], pR = s[5];
  const GasC<double> G(gamma);
  const double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  if (!(rL > 0.0) || !(rR > 0.0) || !(pL > 0.0) || !(pR > 0.0) || G.two_gm1 * (cL + cR) <= uR - uL) {
    target[i] = __int_as_float(0x7fc00000);
    return;
  }
  RiemannInfo info{0, 0, 0, 0};
  NewtonTail<double> nt;
  const double p0 = standard_guess(rL, uL, pL, cL, rR, uR, pR, cR, G);
  const double p = newton_pstar(p0, rL, uL, pL, cL, rR, uR, pR, cR, G, tol, tol, maxit, info, nt);
  const GasC<float> Gf(gamma);
  const float cLf = sqrtf(Gf.g * s[2] / s[0]), cRf = sqrtf(Gf.g * s[5] / s[3]);
  const float ppv = linearised_pstar(s[0], s[1], s[2], cLf, s[3], s[4], s[5], cRf);
  const float pts = two_shock_pstar(s[0], s[1], s[2], s[3], s[4], s[5], ppv, Gf);
  target[i] = (info.fail || !(pts > 0.0f)) ? __int_as_float(0x7fc00000) : (float)log(p / (double)pts);
}

}  // namespace amm

// ============================================================ C ABI
struct amm_mlp {
  double gamma = 5.0 / 3.0;
  cudaStream_t stream = nullptr;
  float* params = nullptr;            // FP32 master parameters [NPARAMS]
  amm::MlpDevice* packed = nullptr;   // BF16 weights for the kernels
  unsigned* status = nullptr;
  // training state
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grads = nullptr;             // [NPARAMS]
  float* partial = nullptr;           // per-CTA gradient partials
  int partial_ctas = 0;
  int64_t adam_t = 0;
  std::string err;
};

namespace {
int mfail(amm_mlp* m, int code, const std::string& msg) {
  if (m) m->err = msg;
  return code;
}
#define MCU(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return mfail(m, AMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t mlp_smem_bytes() { return sizeof(amm::MlpSmem) + 1024; }
size_t train_smem_bytes() { return sizeof(amm::TrainSmem) + 1024; }

int ensure_train(amm_mlp* m, int ctas) {
  if (!m->adam_m) {
    MCU(cudaMalloc(&m->adam_m, sizeof(float) * amm::NPARAMS));
    MCU(cudaMalloc(&m->adam_v, sizeof(float) * amm::NPARAMS));
    MCU(cudaMalloc(&m->grads, sizeof(float) * (amm::NPARAMS + 1)));
    MCU(cudaMemset(m->adam_m, 0, sizeof(float) * amm::NPARAMS));
    MCU(cudaMemset(m->adam_v, 0, sizeof(float) * amm::NPARAMS));
  }
  if (m->partial_ctas < ctas) {
    if (m->partial) cudaFree(m->partial);
    m->partial = nullptr;
    MCU(cudaMalloc(&m->partial, sizeof(float) * (amm::NPARAMS + 1) * (size_t)ctas));
    m->partial_ctas = ctas;
  }
  return AMM_OK;
}

// gradients of the batch into m->grads (device), loss in m->grads[NPARAMS]
int run_grads(amm_mlp* m, const float* x, const float* t, const int* idx, int64_t n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (n + amm::MLP_TILE - 1) / amm::MLP_TILE;
  const int ctas = (int)std::min<int64_t>(tiles, (int64_t)sms);
  int rc = ensure_train(m, ctas);
  if (rc != AMM_OK) return rc;
  amm::k_mlp_grads<<<ctas, amm::MLP_TILE, train_smem_bytes(), m->stream>>>(m->packed, x, t, idx, n, 1.0f / (float)n,
                                                                          m->partial, m->status);
  MCU(cudaGetLastError());
  amm::k_mlp_reduce<<<(amm::NPARAMS + 256) / 256, 256, 0, m->stream>>>(m->partial, ctas, m->grads);
  MCU(cudaGetLastError());
  return AMM_OK;
}
}  // namespace

extern "C" {

int amm_mlp_create(amm_mlp** out, double gamma, void* stream) {
  if (!out || !(gamma > 1.0)) return AMM_ERR_INVALID_ARG;
  *out = nullptr;
  amm_mlp* m = new amm_mlp();
  m->gamma = gamma;
  m->stream = (cudaStream_t)stream;
  auto bail = [&](int rc) {
    if (m->params) cudaFree(m->params);
    if (m->packed) cudaFree(m->packed);
    if (m->status) cudaFree(m->status);
    delete m;
    return rc;
  };
  if (cudaMalloc(&m->params, sizeof(float) * amm::NPARAMS) != cudaSuccess) return bail(AMM_ERR_CUDA);
  if (cudaMalloc(&m->packed, sizeof(amm::MlpDevice)) != cudaSuccess) return bail(AMM_ERR_CUDA);
  if (cudaMalloc(&m->status, sizeof(unsigned)) != cudaSuccess) return bail(AMM_ERR_CUDA);
  if (cudaMemset(m->params, 0, sizeof(float) * amm::NPARAMS) != cudaSuccess) return bail(AMM_ERR_CUDA);
  if (cudaMemset(m->status, 0, sizeof(unsigned)) != cudaSuccess) return bail(AMM_ERR_CUDA);
  if (cudaFuncSetAttribute(amm::k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes()) !=
      cudaSuccess)
    return bail(AMM_ERR_CUDA);
  if (cudaFuncSetAttribute(amm::k_mlp_grads, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem_bytes()) !=
      cudaSuccess)
    return bail(AMM_ERR_CUDA);
  *out = m;
  return AMM_OK;
}

void amm_mlp_destroy(amm_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  void* ptrs[] = {m->params, m->packed, m->status, m->adam_m, m->adam_v, m->grads, m->partial};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

const char* amm_mlp_last_error(const amm_mlp* m) { return m ? m->err.c_str() : "null handle"; }

int amm_mlp_num_params(void) { return amm::NPARAMS; }

int amm_mlp_set_params(amm_mlp* m, const float* params) {
  if (!m || !params) return mfail(m, AMM_ERR_INVALID_ARG, "null argument");
  for (int i = 0; i < amm::NPARAMS; i++)
    if (!std::isfinite(params[i])) return mfail(m, AMM_ERR_INVALID_ARG, "non-finite parameter");
  MCU(cudaMemcpyAsync(m->params, params, sizeof(float) * amm::NPARAMS, cudaMemcpyHostToDevice, m->stream));
  amm::k_mlp_pack<<<1, 256, 0, m->stream>>>(m->params, m->packed);
  MCU(cudaGetLastError());
  MCU(cudaStreamSynchronize(m->stream));
  return AMM_OK;
}

int amm_mlp_get_params(amm_mlp* m, float* params) {
  if (!m || !params) return mfail(m, AMM_ERR_INVALID_ARG, "null argument");
  MCU(cudaMemcpyAsync(params, m->params, sizeof(float) * amm::NPARAMS, cudaMemcpyDeviceToHost, m->stream));
  MCU(cudaStreamSynchronize(m->stream));
  return AMM_OK;
}

int amm_mlp_forward(amm_mlp* m, const float* x_device, int64_t n, float* y_device) {
  if (!m || !x_device || !y_device || n < 1) return mfail(m, AMM_ERR_INVALID_ARG, "bad argument");
  const int64_t tiles = (n + amm::MLP_TILE - 1) / amm::MLP_TILE;
  amm::k_mlp_forward<<<(unsigned)tiles, amm::MLP_TILE, mlp_smem_bytes(), m->stream>>>(m->packed, x_device, n,
                                                                                     y_device, m->status);
  MCU(cudaGetLastError());
  unsigned st = 0;
  MCU(cudaMemcpyAsync(&st, m->status, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
  MCU(cudaStreamSynchronize(m->stream));
  if (st) return mfail(m, AMM_ERR_TIMEOUT, "tensor-core wait timed out");
  return AMM_OK;
}

int amm_mlp_grads(amm_mlp* m, const float* x_device, const float* t_device, const int32_t* idx_device, int64_t n,
                  float* grads, float* loss) {
  if (!m || !x_device || !t_device || n < 1 || !grads) return mfail(m, AMM_ERR_INVALID_ARG, "bad argument");
  int rc = run_grads(m, x_device, t_device, idx_device, n);
  if (rc != AMM_OK) return rc;
  std::vector<float> g(amm::NPARAMS + 1);
  unsigned st = 0;
  MCU(cudaMemcpyAsync(g.data(), m->grads, sizeof(float) * g.size(), cudaMemcpyDeviceToHost, m->stream));
  MCU(cudaMemcpyAsync(&st, m->status, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
  MCU(cudaStreamSynchronize(m->stream));
  if (st) return mfail(m, AMM_ERR_TIMEOUT, "tensor-core wait timed out");
  for (int i = 0; i < amm::NPARAMS; i++) grads[i] = g[i];
  if (loss) *loss = g[amm::NPARAMS];
  return AMM_OK;
}

int amm_mlp_train_step(amm_mlp* m, const float* x_device, const float* t_device, const int32_t* idx_device, int64_t n,
                       float lr, float* loss_device) {
  if (!m || !x_device || !t_device || n < 1 || !(lr > 0.0f)) return mfail(m, AMM_ERR_INVALID_ARG, "bad argument");
  int rc = run_grads(m, x_device, t_device, idx_device, n);
  if (rc != AMM_OK) return rc;
  m->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)m->adam_t), c2 = 1.0f - powf(b2, (float)m->adam_t);
  amm::k_mlp_adam<<<(amm::NPARAMS + 255) / 256, 256, 0, m->stream>>>(m->params, m->grads, m->adam_m, m->adam_v, lr, b1,
                                                                    b2, 1e-8f, c1, c2);
  MCU(cudaGetLastError());
  amm::k_mlp_pack<<<1, 256, 0, m->stream>>>(m->params, m->packed);
  MCU(cudaGetLastError());
  if (loss_device)
    MCU(cudaMemcpyAsync(loss_device, m->grads + amm::NPARAMS, sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
  return AMM_OK;
}

int amm_mlp_sync(amm_mlp* m) {
  if (!m) return AMM_ERR_INVALID_ARG;
  unsigned st = 0;
  MCU(cudaMemcpyAsync(&st, m->status, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
  MCU(cudaStreamSynchronize(m->stream));
  if (st) return mfail(m, AMM_ERR_TIMEOUT, "tensor-core wait timed out");
  return AMM_OK;
}

int amm_mlp_attach(amm_ctx* c, const amm_mlp* m) {
  if (!c || !m) return AMM_ERR_INVALID_ARG;
  if (c->opt.precision != AMM_FP32_LEARNED) {
    c->err = "amm_mlp_attach: the context is not of the FP32 learned form";
    return AMM_ERR_INVALID_ARG;
  }
  if (!c->mlp && cudaMalloc(&c->mlp, sizeof(amm::MlpDevice)) != cudaSuccess) {
    c->err = "amm_mlp_attach: cudaMalloc failed";
    return AMM_ERR_CUDA;
  }
  // the list of faces past the proposal's gate (room for every face)
  if (!c->defer_list && (cudaMalloc((void**)&c->defer_list, sizeof(int2) * (size_t)std::max<int64_t>(c->nf_cap, 1)) !=
                             cudaSuccess ||
                         cudaMalloc((void**)&c->defer_count, sizeof(unsigned)) != cudaSuccess)) {
    c->err = "amm_mlp_attach: cudaMalloc failed";
    return AMM_ERR_CUDA;
  }
  if (cudaMemcpyAsync(c->mlp, m->packed, sizeof(amm::MlpDevice), cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess || amm::prepare_flux_learned() != cudaSuccess) {
    c->err = "amm_mlp_attach: copy failed";
    return AMM_ERR_CUDA;
  }
  c->mlp_loaded = true;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return AMM_OK;
}

int amm_mlp_features(double gamma, int64_t n, const float* states_device, float* x_device, float* pbar_device,
                     float* pts_device, float* ratio_device, void* stream) {
  if (!(gamma > 1.0) || n < 1 || !states_device || !x_device) return AMM_ERR_INVALID_ARG;
  amm::k_mlp_features<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      gamma, n, states_device, x_device, pbar_device, pts_device, ratio_device);
  return cudaGetLastError() == cudaSuccess ? AMM_OK : AMM_ERR_CUDA;
}

int amm_mlp_targets(double gamma, int64_t n, const float* states_device, double tol, float* target_device,
                    void* stream) {
  if (!(gamma > 1.0) || n < 1 || !states_device || !target_device || !(tol > 0.0)) return AMM_ERR_INVALID_ARG;
  amm::k_mlp_targets<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(gamma, n, states_device, tol, 200,
                                                                                   target_device);
  return cudaGetLastError() == cudaSuccess ? AMM_OK : AMM_ERR_CUDA;
}

int amm_riemann_pstar(double gamma, int64_t n, const float* states_device, double tol, float* pstar_device,
                      void* stream) {
  if (!(gamma > 1.0) || n < 1 || !states_device || !pstar_device || !(tol > 0.0)) return AMM_ERR_INVALID_ARG;
  amm::k_riemann_pstar<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(gamma, n, states_device, tol,
                                                                                     200, pstar_device);
  return cudaGetLastError() == cudaSuccess ? AMM_OK : AMM_ERR_CUDA;
}

}  // extern "C"
