// Face fluxes of the FP32 forms (A5-A7: face velocity, MUSCL-Hancock
// extrapolation in the face frame, exact Riemann solve, flux of the moving
// face; Sec. 3.3) as a persistent kernel over chunks of faces.
//
// What bounds it: each face gathers two cell records (W, {P, s - r} and four
// gradient vectors, 96 bytes each) from scattered cells.  A warp's load of
// one 16-byte piece of 32 scattered records touches 32 cache lines, and the
// L1 data pipe returns one line per cycle, so with 16-byte loads the gathers
// alone kept that pipe 70% busy.  Here every record is read with 32-byte
// (256-bit) loads: the same lines in half the instructions, so half the
// wavefronts.  (Staging the records in shared memory was measured and is
// slower: per-thread asynchronous copies write shared memory once per
// scattered line, and bulk-copy (TMA) gathers of 32- and 64-byte records
// wait on the copy engine's latency.)
//
// Each CTA of B threads walks a contiguous range of B-face chunks (each chunk
// inside one face tile, so inside one box), one face per thread and chunk.
// The chunk's tile record is read two chunks ahead and the face's cell
// indices one chunk ahead, so the cell gathers do not wait behind index
// loads.  There is no barrier inside the loop: the Newton statistics are
// kept per warp in shared memory and added to the device totals once per
// CTA; the running maxima of |A F| per component (of the current box) are
// kept per thread and reduced over the warp when the box changes.
//
// Static mesh (STATIC): the face frame is the lab frame, so a cell's
// half-step prediction W - (dt/2) A(W) grad W is the same for all its faces;
// the gradient kernel writes it once per cell (cwp) and a face only
// extrapolates the two predicted records to its centroid, instead of
// repeating the prediction on each of a cell's ~15 faces.
//
// Learned form (LEARN): a face whose Riemann problem would take the proposal
// (the linearised star pressure above PROPOSAL_GATE times the larger side
// pressure) is not solved here; it is appended, warp by warp, to a list that
// k_flux_deferred (flux_learned.cu) completes with the tensor-core proposal,
// so this kernel keeps its occupancy and the network runs only on the faces
// that use it.
#include <cuda_runtime.h>

#include "hydro.cuh"
#include "learned.cuh"

namespace amm {

// CTAs per SM each shape is compiled for (launch bounds, and so registers)
template <int B>
constexpr int chunk_ctas_per_sm() {
  return B == 256 ? 3 : 7;
}

// per warp: iteration histogram, statistics sums
template <int B>
struct ChunkSmem {
  unsigned hist[B / 32][16];
  unsigned red[B / 32][8];
};

// a cell's record: {rho, v}, {P, s - r} (32 bytes: from cw, or the
// predicted record from cwp) and its gradients (64); A from Aw or Apw
template <bool ENT>
__device__ __forceinline__ CellRec<float> load_rec256(const HydroView<float>& v, const R4<float>* rec,
                                                     const float* A, int i) {
  CellRec<float> r;
  ldg256(rec + 2 * (size_t)i, r.W, r.Pc);
  ldg256(v.grad + 4 * (size_t)i, r.g0, r.g1);
  ldg256(v.grad + 4 * (size_t)i + 2, r.g2, r.g3);
  if constexpr (ENT) {
    r.A = A[i];
    r.gA = v.gradA[i];
  }
  return r;
}

// face of this thread in chunk c of tile T (FACE_TILE / B chunks per tile);
// faces past the tile's end take the tile's first face (in bounds; their
// results are not stored)
template <int B>
__device__ __forceinline__ int chunk_face(int c, const Tile& T, bool& valid) {
  const int k = T.begin + (c % (FACE_TILE / B)) * B + (int)threadIdx.x;
  valid = k < T.end;
  return valid ? k : T.begin;
}

template <int B, bool ENT, bool LEARN, bool STATIC>
__global__ void __launch_bounds__(B, chunk_ctas_per_sm<B>()) k_flux_chunks(HydroView<float> v, int nchunks, int per_cta,
                                                                          FluxDefer defer) {
  constexpr int CPT = FACE_TILE / B;   // chunks per face tile
  __shared__ ChunkSmem<B> sm;
  constexpr int NM = ENT ? 6 : 5;
  const unsigned full = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int c0 = blockIdx.x * per_cta;
  const int c1 = min(nchunks, c0 + per_cta);
  if (c0 >= c1) return;   // the whole CTA leaves together
  if (lane < 16) sm.hist[warp][lane] = 0u;
  if (lane < 8) sm.red[warp][lane] = 0u;
  __syncwarp();
  const bool fixed = v.fixed_acc != 0;
  // each thread's running maxima of |A F| per component (of the current box),
  // reduced over the warp when the box changes
  unsigned fm[NM];
#pragma unroll
  for (int a = 0; a < NM; a++) fm[a] = 0u;

  // tiles of chunks c0 and c0+1, cell indices of c0
  Tile T0 = v.ftiles[c0 / CPT];
  Tile T1 = (c0 + 1 < c1) ? v.ftiles[(c0 + 1) / CPT] : T0;
  bool vtmp;
  int2 L0 = v.lr[chunk_face<B>(c0, T0, vtmp)];
  // half the box's step, in FP32 (the FP64 arithmetic of box_dt runs on the
  // narrow FP64 pipe, so once per box, not per face)
  int hbox = T0.box;
  float hdt = (float)(0.5 * box_dt(v, hbox));

  for (int c = c0; c < c1; c++) {
    const bool more1 = c + 1 < c1;
    // tile of c+2, cell indices of c+1 (their loads overlap this chunk)
    const Tile T2 = (c + 2 < c1) ? v.ftiles[(c + 2) / CPT] : T1;
    const int2 L1 = more1 ? v.lr[chunk_face<B>(c + 1, T1, vtmp)] : L0;
    bool valid;
    const int k = chunk_face<B>(c, T0, valid);
    if (T0.box != hbox) {
      hbox = T0.box;
      hdt = (float)(0.5 * box_dt(v, hbox));
    }
    FaceWork<float> f;
    {
      R4<float> G0, G1;
      ldg256(v.fgeo + 2 * (size_t)k, G0, G1);
      if constexpr (STATIC) {
        // the cells' half-step predicted records (gradient kernel)
        const CellRec<float> pL = load_rec256<ENT>(v, v.cwp, v.Apw, L0.x);
        const CellRec<float> pR = load_rec256<ENT>(v, v.cwp, v.Apw, L0.y);
        float AL = 0.0f, AR = 0.0f;
        if constexpr (ENT) {
          AL = v.Aw[L0.x];
          AR = v.Aw[L0.y];
        }
        face_prepare_pred<float, ENT>(v, k, valid, L0, G0, G1, pL, pR, AL, AR, f);
      } else {
        const CellRec<float> recL = load_rec256<ENT>(v, v.cw, v.Aw, L0.x);
        const CellRec<float> recR = load_rec256<ENT>(v, v.cw, v.Aw, L0.y);
        face_prepare_rec<float, ENT>(v, k, valid, hdt, hdt, L0, G0, G1, recL, recR, f);
      }
    }
    bool mine = valid;
    float cs[3];   // c_L, c_R and the linearised star pressure, for the gate and the solver
    if constexpr (LEARN) {
      // faces that take the proposal go to the deferred list, warp by warp
      const float g = v.gas.g;
      cs[0] = sqrtf(g * f.WppL[4] / f.WppL[0]);
      cs[1] = sqrtf(g * f.WppR[4] / f.WppR[0]);
      cs[2] = linearised_pstar(f.WppL[0], f.uL, f.WppL[4], cs[0], f.WppR[0], f.uR, f.WppR[4], cs[1]);
      const bool need = valid && cs[2] > PROPOSAL_GATE * fmaxf(f.WppL[4], f.WppR[4]);
      const unsigned nb = __ballot_sync(full, need);
      if (nb) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(defer.count, (unsigned)__popc(nb));
        base = __shfl_sync(full, base, 0);
        if (need) {
          const unsigned pos = base + (unsigned)__popc(nb & ((1u << lane) - 1u));
          if (pos < defer.capacity) defer.list[pos] = make_int2(k, T0.box);
        }
      }
      mine = valid && !need;
      f.valid = mine;
      if (need) {
        // the lane's solve is discarded: give it a problem that converges at
        // once (equal states) so that it does not hold up its warp
#pragma unroll
        for (int a = 0; a < 5; a++) f.WppR[a] = f.WppL[a];
        f.uR = f.uL;
        cs[1] = cs[0];
        cs[2] = f.WppL[4];
      }
    }
    FaceOut o;
    face_finish_core<float, ENT>(v, f, false, 0.0f, o, LEARN, cs);
    if constexpr (STATIC) {
#pragma unroll
      for (int a = 0; a < NM; a++) fm[a] = max(fm[a], o.m[a]);
    } else {
      // the moving-mesh instantiation holds more live values: a warp
      // reduction per chunk spills less than five private maxima (measured
      // 4.6% faster at 64^3)
#pragma unroll
      for (int a = 0; a < NM; a++) {
        const unsigned r = __reduce_max_sync(full, o.m[a]);
        fm[a] = max(fm[a], r);
      }
    }
    // Newton statistics of the warp: the iteration histogram (the lanes with
    // equal counts found by one match; the lowest of them adds their number,
    // so the lanes that write hold distinct bins), sums and flags
    const unsigned act = __ballot_sync(full, mine);
    {
      const unsigned key = mine ? (o.iters < 15u ? o.iters : 15u) : 0xffffffffu;
      const unsigned m = __match_any_sync(full, key);
      if (mine && lane == __ffs(m) - 1) sm.hist[warp][key] += __popc(m);
    }
    const unsigned sit = __reduce_add_sync(full, o.iters);
    const unsigned smx = __reduce_max_sync(full, o.iters);
    if (lane == 0) {
      sm.red[warp][0] += __popc(act);
      sm.red[warp][1] += sit;
      sm.red[warp][6] = max(sm.red[warp][6], smx);
    }
    if (__any_sync(full, o.guard || o.vacuum || o.fail || o.fallback)) {
      const unsigned g = __popc(__ballot_sync(full, o.guard)), va = __popc(__ballot_sync(full, o.vacuum));
      const unsigned fa = __popc(__ballot_sync(full, o.fail)), fb = __popc(__ballot_sync(full, o.fallback));
      if (lane == 0) {
        sm.red[warp][2] += g;
        sm.red[warp][3] += va;
        sm.red[warp][4] += fa;
        sm.red[warp][5] += fb;
      }
      if (o.fail) atomicOr(v.box_status + T0.box, (unsigned)ST_NEWTON_CAP);
    }
    // the box's maxima at its last chunk of this CTA
    if (fixed && (!more1 || T1.box != T0.box)) {
#pragma unroll
      for (int a = 0; a < NM; a++) {
        const unsigned r = __reduce_max_sync(full, fm[a]);
        if (lane == 0 && r) atomicMax(v.fmax_bits + FMAX_STRIDE * T0.box + a, r);
        fm[a] = 0u;
      }
    }
    T0 = T1;
    T1 = T2;
    L0 = L1;
  }
  // one set of global atomics per CTA for the statistics
  __syncthreads();
  if (t < 16) {
    unsigned h = 0;
    for (int w = 0; w < B / 32; w++) h += sm.hist[w][t];
    if (h) atomicAdd(&v.stats->hist[t], (unsigned long long)h);
  } else if (t == 16) {
    unsigned long long a[6] = {0, 0, 0, 0, 0, 0};
    unsigned mx = 0;
    for (int w = 0; w < B / 32; w++) {
      for (int q = 0; q < 6; q++) a[q] += sm.red[w][q];
      mx = max(mx, sm.red[w][6]);
    }
    stats_add(v.stats, v.box_status, -1, a[0], a[1], (unsigned)a[2], (unsigned)a[3], (unsigned)a[4], (unsigned)a[5],
              mx);
  }
}

template <int B, bool ENT, bool LEARN, bool STATIC>
static cudaError_t launch_chunks(amm_ctx* c, const HydroView<float>& v, const FluxDefer& defer) {
  auto kern = k_flux_chunks<B, ENT, LEARN, STATIC>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, 0)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int nchunks = (FACE_TILE / B) * c->n_ftiles;
  if (nchunks == 0) return cudaSuccess;
  const int slots = per_sm * sms;
  const int per_cta = (nchunks + slots - 1) / slots;
  const int grid = (nchunks + per_cta - 1) / per_cta;
  kern<<<grid, B, 0, c->stream>>>(v, nchunks, per_cta, defer);
  return cudaGetLastError();
}

template <int B, bool STATIC>
static cudaError_t launch_chunks_s(amm_ctx* c, const HydroView<float>& v, bool learn, const FluxDefer& defer) {
  const bool ent = c->opt.entropy != 0;
  if (learn)
    return ent ? launch_chunks<B, true, true, STATIC>(c, v, defer) : launch_chunks<B, false, true, STATIC>(c, v, defer);
  return ent ? launch_chunks<B, true, false, STATIC>(c, v, defer) : launch_chunks<B, false, false, STATIC>(c, v, defer);
}

template <int B>
static cudaError_t launch_chunks_b(amm_ctx* c, const HydroView<float>& v, bool learn, const FluxDefer& defer) {
  // a static mesh (no mesh velocity anywhere) has its own instantiation
  if (c->opt.mesh_motion == AMM_EULERIAN) return launch_chunks_s<B, true>(c, v, learn, defer);
  return launch_chunks_s<B, false>(c, v, learn, defer);
}

cudaError_t launch_flux_chunks(amm_ctx* c, const HydroView<float>& v, bool learn, const FluxDefer& defer) {
  return c->flux_block == 256 ? launch_chunks_b<256>(c, v, learn, defer) : launch_chunks_b<128>(c, v, learn, defer);
}

}  // namespace amm
