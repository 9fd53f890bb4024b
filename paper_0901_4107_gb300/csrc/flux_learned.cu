// Face fluxes of the FP32 learned form with the proposal network on the
// tensor cores.  A CTA of H x 128 threads handles H x 128 prepared faces at a
// time: every thread whose face passes the gate writes the normalised
// features as row (t mod 128) of the BF16 operand of its group, one thread
// issues the tensor-core layers of all groups (tcgen05, FP32 accumulators in
// tensor memory: group h owns columns 64h..64h+63, reused by both layers),
// every thread reads its row back, forms p0 = p_TS exp(y) and runs the exact
// Riemann solver from it.  Newton still iterates to the same tolerance, so
// the result depends on the network only through the iteration count.
//
// Two kernels use it: k_flux_deferred (H = 1: the faces that the plain FP32
// flux kernel, flux_chunks.cu, found past the gate and listed) and
// k_step_persistent_learned (H = 2, the whole step as one cooperative
// launch, the batched-ensemble form).  Both run the same per-face arithmetic;
// compiled under different register budgets, they may contract a
// multiply-add differently, so the two step modes agree to FP32 rounding.
#include <cuda_runtime.h>

#include "hydro.cuh"
#include "learned.cuh"
#include "persistent.cuh"
#include "tc.cuh"

namespace amm {

constexpr int LT = 128;  // faces per MMA group = MMA rows
// CTAs of k_flux_deferred per SM (launch bounds and grid); their tensor memory
// (64 columns each) must fit the SM's 512
constexpr int LEARNED_CTAS_PER_SM = 4;
static_assert(LEARNED_CTAS_PER_SM * 64 <= 512, "tensor-memory columns of the co-resident CTAs");

template <int H>
struct LearnedSmem {
  alignas(1024) uint8_t a1[H][LT * 16 * 2];
  alignas(1024) uint8_t a2[H][LT * MLP_HID * 2];
  alignas(1024) uint8_t b1[MLP_HID * 16 * 2];
  alignas(1024) uint8_t b2[MLP_HID * MLP_HID * 2];
  float bias1[MLP_HID], bias2[MLP_HID], w3[MLP_HID], bias3;
  float hdt;
  uint64_t mbar;
  uint32_t tmem;
  uint32_t ok;
};

template <int H>
__host__ __device__ constexpr size_t learned_smem_bytes() {
  return sizeof(LearnedSmem<H>) + 1024;  // + alignment slack of the dynamic block
}

template <int H>
__device__ __forceinline__ LearnedSmem<H>& learned_smem_ref(uint8_t* raw) {
  return *reinterpret_cast<LearnedSmem<H>*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
}

// SiLU from one hardware tanh: z sigma(z) = z/2 (1 + tanh(z/2)); the
// proposal only seeds Newton, so the approximate tanh is accurate enough
__device__ __forceinline__ float silu_fast(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return 0.5f * z * (1.0f + t);
}

// tensor-memory allocation (64 H columns), mbarrier, weights into shared
// memory in the K-major core-matrix layout of the MMA operands
template <int H>
__device__ __forceinline__ void learned_setup(LearnedSmem<H>& s, const MlpDevice* M) {
  const int t = threadIdx.x;
  if (t < 32) tc::tmem_alloc(&s.tmem, 64 * H);
  if (t == 0) {
    tc::mbar_init(&s.mbar, 1);
    s.ok = 1;
  }
  // eight consecutive k of one row are one 16-byte row segment of a core
  // matrix: 16-byte loads and stores, all independent
  const uint4* w1 = reinterpret_cast<const uint4*>(M->W1);
  const uint4* w2 = reinterpret_cast<const uint4*>(M->W2);
  for (int i = t; i < MLP_HID * 16 / 8; i += H * LT)
    *reinterpret_cast<uint4*>(s.b1 + tc::kmajor_offset(i / 2, 8 * (i % 2), 16)) = w1[i];
  for (int i = t; i < MLP_HID * MLP_HID / 8; i += H * LT)
    *reinterpret_cast<uint4*>(s.b2 + tc::kmajor_offset(i / 8, 8 * (i % 8), MLP_HID)) = w2[i];
  if (t < MLP_HID) {
    s.bias1[t] = M->b1[t];
    s.bias2[t] = M->b2[t];
    s.w3[t] = __bfloat162float(M->W3[t]);
  }
  if (t == 0) s.bias3 = M->b3;
}

// The proposal for the prepared face f, by all H x 128 threads of the CTA:
// whether this face takes it (`use`) and the starting value p_TS exp(y).
// A face takes it when its compression is strong: the linearised estimate
// above PROPOSAL_GATE times the larger pressure (which also places it in the
// two-shock branch of the standard guess).  If no face of the CTA does, the
// network is skipped.
template <int H>
__device__ __forceinline__ void learned_guess(const HydroView<float>& v, LearnedSmem<H>& s, const FaceWork<float>& f,
                                              uint32_t& phase, bool& use, float& guess) {
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int h = t / LT;       // MMA group of this thread
  const int row = t % LT;     // its row in the group's tiles
  const int quad = warp & 3;  // tensor-memory lane quadrant this warp may read
  const uint32_t idesc = tc::make_idesc(LT, MLP_HID);
  const float g = v.gas.g;
  const float rb = 0.5f * (f.WppL[0] + f.WppR[0]);
  const float pb = 0.5f * (f.WppL[4] + f.WppR[4]);
  bool need = false;
  float pts = pb;
  {
    const float cL = sqrtf(g * f.WppL[4] / f.WppL[0]), cR = sqrtf(g * f.WppR[4] / f.WppR[0]);
    const float ppv = linearised_pstar(f.WppL[0], f.uL, f.WppL[4], cL, f.WppR[0], f.uR, f.WppR[4], cR);
    need = f.valid && ppv > PROPOSAL_GATE * fmaxf(f.WppL[4], f.WppR[4]);
    if (need) pts = two_shock_pstar(f.WppL[0], f.uL, f.WppL[4], f.WppR[0], f.uR, f.WppR[4], ppv, v.gas);
  }
  use = false;
  guess = 0.0f;
  if (!__syncthreads_or(need)) return;
  // normalised features (the network's input)
  const float icb = rsqrtf(g * pb / rb);
  {
    const float irb = 1.0f / rb, ipb = 1.0f / pb;
    float x[16] = {__logf(f.WppL[0] * irb), __logf(f.WppL[4] * ipb), f.uL * icb, __logf(f.WppR[0] * irb),
                   __logf(f.WppR[4] * ipb), f.uR * icb, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    tc::st_bf16x8(s.a1[h], tc::kmajor_offset(row, 0, 16), x);
    tc::st_bf16x8(s.a1[h], tc::kmajor_offset(row, 8, 16), x + 8);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < H; q++)
      tc::mma_bf16(s.tmem + 64 * q, tc::kmajor_desc(tc::smem_addr(s.a1[q]), 16),
                   tc::kmajor_desc(tc::smem_addr(s.b1), 16), idesc, false);
    tc::mma_commit(&s.mbar);
  }
  if (!tc::mbar_wait(&s.mbar, phase)) s.ok = 0;
  phase ^= 1u;
  tc::fence_after_sync();
#pragma unroll
  for (int c = 0; c < 4; c++) {
    float z[16];
    tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, quad, 64 * h + 16 * c), z);
#pragma unroll
    for (int j = 0; j < 16; j++) z[j] = silu_fast(z[j] + s.bias1[16 * c + j]);
    tc::st_bf16x8(s.a2[h], tc::kmajor_offset(row, 16 * c, MLP_HID), z);
    tc::st_bf16x8(s.a2[h], tc::kmajor_offset(row, 16 * c + 8, MLP_HID), z + 8);
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < H; q++)
#pragma unroll
      for (int kb = 0; kb < MLP_HID / 16; kb++)
        tc::mma_bf16(s.tmem + 64 * q, tc::kmajor_desc(tc::smem_addr(s.a2[q]) + 256 * kb, MLP_HID),
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
    tc::tmem_ld16(tc::tmem_lane_addr(s.tmem, quad, 64 * h + 16 * c), z);
#pragma unroll
    for (int j = 0; j < 16; j++) y += s.w3[16 * c + j] * silu_fast(z[j] + s.bias2[16 * c + j]);
  }
  y = fminf(fmaxf(y, -30.0f), 30.0f);
  use = need && s.ok != 0;  // after a timed-out wait, fall back to the standard guess
  guess = pts * __expf(y);
}

// H x 128 faces starting at `first` (faces at or past `end` are padding)
template <int H, bool ENT>
__device__ __forceinline__ void learned_faces(const HydroView<float>& v, LearnedSmem<H>& s, const Tile& tile,
                                              int first, uint32_t& phase) {
  const int t = threadIdx.x;
  const int k0 = first + t;
  const bool valid = k0 < tile.end;
  if (t == 0) s.hdt = (float)(0.5 * box_dt(v, tile.box));
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  FaceWork<float> f;
  face_prepare_step<float, ENT>(v, valid ? k0 : tile.begin, valid, s.hdt, f);
  bool use;
  float guess;
  learned_guess<H>(v, s, f, phase, use, guess);
  face_finish<float, H * LT, ENT>(v, f, tile.box, min(H * LT, tile.end - first), use, guess);
}

template <int H>
__device__ __forceinline__ void learned_teardown(const HydroView<float>& v, LearnedSmem<H>& s) {
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && !s.ok) atomicOr(&v.stats->status, (unsigned)ST_TIMEOUT);
  if (threadIdx.x < 32) tc::tmem_dealloc(s.tmem, 64 * H);
}

// The faces the plain FP32 kernel (k_flux_chunks, flux_chunks.cu) deferred: each list entry
// {face, box} is prepared again from global memory, takes the proposal and
// is solved; 128 entries per CTA at a time.  CTAs beyond the list's length
// leave before touching tensor memory, so with an empty list the launch
// costs only its CTAs' start.
template <bool ENT>
__global__ void __launch_bounds__(LT, LEARNED_CTAS_PER_SM) k_flux_deferred(HydroView<float> v, FluxDefer d) {
  const unsigned count = min(*d.count, d.capacity);
  const unsigned groups = (count + LT - 1) / LT;
  if (blockIdx.x >= groups) return;
  extern __shared__ uint8_t smem_raw[];
  LearnedSmem<1>& s = learned_smem_ref<1>(smem_raw);
  learned_setup<1>(s, (const MlpDevice*)v.mlp);
  __shared__ unsigned hist[LT / 32][16];
  __shared__ unsigned red[LT / 32][8];
  constexpr int NM = ENT ? 6 : 5;
  const unsigned full = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (lane < 16) hist[warp][lane] = 0u;
  __syncwarp();
  unsigned s_faces = 0, s_iters = 0, s_guard = 0, s_vac = 0, s_fail = 0, s_fb = 0, s_max = 0;
  uint32_t phase = 0;
  for (unsigned gi = blockIdx.x; gi < groups; gi += gridDim.x) {
    const unsigned e = gi * LT + (unsigned)t;
    const bool valid = e < count;
    const int2 kb = d.list[valid ? e : gi * LT];
    const float hdt = (float)(0.5 * box_dt(v, kb.y));
    FaceWork<float> f;
    face_prepare_step<float, ENT>(v, kb.x, valid, hdt, f);
    bool use;
    float guess;
    learned_guess<1>(v, s, f, phase, use, guess);
    FaceOut o;
    face_finish_core<float, ENT>(v, f, use, guess, o);
    if (v.fixed_acc) {
      // the list is filled warp by warp from one chunk, so a warp's entries
      // normally share a box
      const int b0 = __shfl_sync(full, kb.y, 0);
      if (__all_sync(full, kb.y == b0)) {
#pragma unroll
        for (int a = 0; a < NM; a++) {
          const unsigned r = __reduce_max_sync(full, o.m[a]);
          if (lane == 0 && r) atomicMax(v.fmax_bits + FMAX_STRIDE * b0 + a, r);
        }
      } else if (valid) {
#pragma unroll
        for (int a = 0; a < NM; a++)
          if (o.m[a]) atomicMax(v.fmax_bits + FMAX_STRIDE * kb.y + a, o.m[a]);
      }
    }
    const unsigned act = __ballot_sync(full, valid);
    {
      // the lanes with equal counts by one match; the lowest adds their number
      const unsigned key = valid ? (o.iters < 15u ? o.iters : 15u) : 0xffffffffu;
      const unsigned m = __match_any_sync(full, key);
      if (valid && lane == __ffs(m) - 1) hist[warp][key] += __popc(m);
    }
    s_faces += __popc(act);
    s_iters += __reduce_add_sync(full, o.iters);
    s_max = max(s_max, __reduce_max_sync(full, o.iters));
    s_guard += __popc(__ballot_sync(full, o.guard));
    s_vac += __popc(__ballot_sync(full, o.vacuum));
    s_fail += __popc(__ballot_sync(full, o.fail));
    s_fb += __popc(__ballot_sync(full, o.fallback));
    if (o.fail) atomicOr(v.box_status + kb.y, (unsigned)ST_NEWTON_CAP);
  }
  if (lane == 0) {
    red[warp][0] = s_faces;
    red[warp][1] = s_iters;
    red[warp][2] = s_guard;
    red[warp][3] = s_vac;
    red[warp][4] = s_fail;
    red[warp][5] = s_fb;
    red[warp][6] = s_max;
  }
  __syncthreads();
  if (t < 16) {
    unsigned h = 0;
    for (int w = 0; w < LT / 32; w++) h += hist[w][t];
    if (h) atomicAdd(&v.stats->hist[t], (unsigned long long)h);
  } else if (t == 16) {
    unsigned long long a[6] = {0, 0, 0, 0, 0, 0};
    unsigned mx = 0;
    for (int w = 0; w < LT / 32; w++) {
      for (int q = 0; q < 6; q++) a[q] += red[w][q];
      mx = max(mx, red[w][6]);
    }
    stats_add(v.stats, v.box_status, -1, a[0], a[1], (unsigned)a[2], (unsigned)a[3], (unsigned)a[4], (unsigned)a[5],
              mx);
  }
  learned_teardown<1>(v, s);
}

// the whole step in one cooperative launch (see persistent.cuh), with the
// flux phase on whole 256-face tiles, two MMA groups per CTA
constexpr int PL_H = FACE_TILE / LT;
static_assert(PL_H * LT == CELL_TILE, "the persistent CTA covers one face tile and one cell tile");

template <bool ENT>
__global__ void __launch_bounds__(CELL_TILE) k_step_persistent_learned(HydroView<float> v, unsigned* bar) {
  extern __shared__ uint8_t smem_raw[];
  LearnedSmem<PL_H>& s = learned_smem_ref<PL_H>(smem_raw);
  learned_setup<PL_H>(s, (const MlpDevice*)v.mlp);
  if (v.pred) {
    for (int wi = blockIdx.x; wi < v.n_ctiles; wi += gridDim.x) courant_item<float>(v, wi);
    grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  }
  const int n_grad = v.n_ctiles * 4;
  for (int wi = blockIdx.x; wi < n_grad; wi += gridDim.x) grad_item<float, 4, ENT>(v, wi);
  grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  uint32_t phase = 0;
  for (int wi = blockIdx.x; wi < v.n_ftiles; wi += gridDim.x) {
    const Tile tile = v.ftiles[wi];
    learned_faces<PL_H, ENT>(v, s, tile, tile.begin, phase);
  }
  grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  for (int wi = blockIdx.x; wi < v.n_ctiles; wi += gridDim.x) update_item<float, 1, ENT>(v, wi);
  grid_barrier(bar, bar + 1, gridDim.x, &v.stats->status);
  for (int b = blockIdx.x; b < v.nboxes; b += gridDim.x) finish_item<float, CELL_TILE>(v, b, 1);
  learned_teardown<PL_H>(v, s);
}

// Tensor memory is 512 columns per SM and an allocation waits until enough
// are free; the persistent kernel keeps its 128 columns until it ends, so at
// most four of its CTAs may share an SM.  Its shared-memory block alone rules
// out a fifth (GB300: 228 KB of shared memory per SM).
static_assert(5 * learned_smem_bytes<PL_H>() > 228 * 1024, "more than 4 persistent learned CTAs could share an SM");
static_assert(4 * 64 * PL_H <= 512, "tensor-memory columns of 4 co-resident CTAs");

cudaError_t prepare_flux_learned() {
  // the largest shared-memory carveout, so that the CTAs the launches assume
  // per SM fit (the occupancy of the cooperative launch is computed with it)
  for (const void* k : {(const void*)k_flux_deferred<false>, (const void*)k_flux_deferred<true>,
                        (const void*)k_step_persistent_learned<false>, (const void*)k_step_persistent_learned<true>}) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaFuncSetAttribute(k_flux_deferred<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)learned_smem_bytes<1>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_deferred<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)learned_smem_bytes<1>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_persistent_learned<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)learned_smem_bytes<PL_H>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_persistent_learned<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)learned_smem_bytes<PL_H>());
  return e;
}

// the learned form's flux phase: the plain FP32 kernel, which lists the
// faces past the gate, then the deferred kernel on the list
cudaError_t launch_flux_learned(amm_ctx* c, const HydroView<float>& v) {
  if (!c->mlp || !c->defer_list || !c->defer_count) return cudaErrorInvalidValue;
  FluxDefer d;
  d.list = c->defer_list;
  d.count = c->defer_count;
  d.capacity = (unsigned)c->nf_cap;
  cudaError_t e = cudaMemsetAsync(c->defer_count, 0, sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return e;
  if ((e = launch_flux_chunks(c, v, true, d)) != cudaSuccess) return e;
  int dev = 0, sms = 148;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  auto kern = c->opt.entropy ? k_flux_deferred<true> : k_flux_deferred<false>;
  // enough CTAs for a list of every face; the ones past its length leave
  const int groups = (int)std::min<int64_t>((c->nf + LT - 1) / LT, (int64_t)LEARNED_CTAS_PER_SM * sms);
  kern<<<std::max(groups, 1), LT, learned_smem_bytes<1>(), c->stream>>>(v, d);
  return cudaGetLastError();
}

cudaError_t launch_step_persistent_learned(amm_ctx* c, double cfl) {
  if (!c->mlp) return cudaErrorInvalidValue;
  auto v = make_view<float>(c, cfl);
  v.update_lanes = 1;
  cudaError_t e = cudaMemsetAsync(c->cour_bits, 0xff, sizeof(unsigned long long) * c->nboxes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->fmax_bits, 0, sizeof(unsigned) * FMAX_STRIDE * c->nboxes, c->stream);
  if (e != cudaSuccess) return e;
  const size_t smem = learned_smem_bytes<PL_H>();
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  auto kern = c->opt.entropy ? k_step_persistent_learned<true> : k_step_persistent_learned<false>;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CELL_TILE, smem)) != cudaSuccess) return e;
  if (per_sm < 1 || per_sm > 4) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(per_sm * sms));
  cfg.blockDim = dim3(CELL_TILE);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, v, c->barrier);
}

}  // namespace amm
