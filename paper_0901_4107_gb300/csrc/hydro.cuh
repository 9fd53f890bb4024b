// Hydro kernels of one update step, templated on the bulk arithmetic type
// (double: FP64 form; float: FP32 form with FP64 accumulation, FP64 Newton
// guard and FP64 sums).  Instantiated in hydro_f64.cu and hydro_f32.cu.
//
//  k_primitives   A1  Q -> W                                  (Sec. 3, step 2)
//  k_gradients    A2+A3+A4  Voronoi gradient (eq. eqngrad2), slope limiter,
//                 per-box Courant minimum (eq. EqnTiStep)     (Sec. 3.1, 7.1)
//  k_flux         A5+A6+A7  face velocity, MUSCL-Hancock extrapolation in the
//                 face frame, exact Riemann solve, flux of the moving face
//                                                             (Sec. 3.3)
//  k_update       A8+A1+A9  signed gather of face fluxes in FP64 (no atomics),
//                 new primitives, per-tile conservation sums  (eq. eqnupdate)
//  k_finish       per-box totals from the tile sums, time step record
//
// One thread per cell (gradients, update) or per face (flux); one CTA per
// tile, each tile inside one box.
#pragma once

#include <cuda_runtime.h>

#include "amm_internal.cuh"
#include "riemann.cuh"

namespace amm {

template <typename real>
__device__ __forceinline__ double box_dt(const HydroView<real>& v, int b) {
  if (v.cfl > 0.0) return v.cfl * __longlong_as_double((long long)v.cour_bits[b]);
  return v.dt_box[b];
}

// 32 bytes of FP32 data from global memory that no thread writes during the
// kernel (32-byte aligned): one 256-bit load.  A warp's gather of 32
// scattered records costs one L1 wavefront per record for each load
// instruction, so one 32-byte load costs half as many as two 16-byte loads.
__device__ __forceinline__ void ldg256(const void* p, R4<float>& a, R4<float>& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// the same for FP64 data: two 32-byte halves of a 64-byte record
__device__ __forceinline__ void ldg256(const void* p, R4<double>& a) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a.x), "=d"(a.y), "=d"(a.z), "=d"(a.w) : "l"(p));
}

// ------------------------------------------------------------------ A1
// Returns P.  The FP32 form keeps only the thermal-energy difference
// E - |p|^2/(2m) in FP64 (it cancels when the flow is supersonic); the FP64
// form is FP64 throughout.
template <typename real>
__device__ __forceinline__ real prims_from_Q(const HydroView<real>& v, int i, double m, double px, double py,
                                             double pz, double E) {
  R4<real> w;
  real P;
  if constexpr (sizeof(real) == 8) {
    const double iV = v.cgeo[i].x;
    const double im = 1.0 / m;
    const double rho = m * iV;
    const double vx = px * im, vy = py * im, vz = pz * im;
    P = (v.gamma - 1.0) * (E * iV - 0.5 * rho * (vx * vx + vy * vy + vz * vz));
    w.x = rho; w.y = vx; w.z = vy; w.w = vz;
  } else {
    const float iV = v.cgeo[i].x;
    const float mf = (float)m;
    const float im = 1.0f / mf;
    const double kin = (px * px + py * py + pz * pz) * (double)(0.5f * im);
    P = v.gas.gm1 * ((float)(E - kin) * iV);
    w.x = mf * iV; w.y = (float)px * im; w.z = (float)py * im; w.w = (float)pz * im;
  }
  v.cw[2 * (size_t)i] = w;
  reinterpret_cast<real*>(v.cw + 2 * (size_t)i + 1)[0] = P;   // .x; s - r stays in .yzw
  return P;
}

template <typename real>
__global__ void k_primitives(HydroView<real> v, unsigned long long* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double m = v.Q[i], px = v.Q[v.n + i], py = v.Q[2 * (size_t)v.n + i], pz = v.Q[3 * (size_t)v.n + i];
  const double E = v.Q[4 * (size_t)v.n + i];
  const real P = prims_from_Q(v, i, m, px, py, pz, E);
  if (v.entropy) v.Aw[i] = (real)(v.S[i] / m);
  if (bad && (!(m > 0.0) || !(P > (real)0))) atomicAdd(bad, 1ull);
}

// ------------------------------------------------------------ A2+A3+A4
// G consecutive lanes share a cell: lane l takes the cell's incidences l,
// l+G, ...; partial sums, extrema and limiter minima are combined with
// butterfly shuffles inside the lane group, so every lane ends with the
// cell's values and lanes split the gradient store.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
template <int G, typename T>
__device__ __forceinline__ T group_max(T x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const T y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}
template <int G, typename T>
__device__ __forceinline__ T group_min(T x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const T y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y < x ? y : x;
  }
  return x;
}

// Mesh velocity of cell i for the Courant step and the cold-flow criterion
template <typename real>
__device__ __forceinline__ void mesh_velocity(const HydroView<real>& v, int i, const R4<real>& Wi, real* w) {
  w[0] = w[1] = w[2] = (real)0;
  if (v.mode == AMM_LAGRANGIAN) {
    w[0] = Wi.y; w[1] = Wi.z; w[2] = Wi.w;
  } else if (v.mode == AMM_EXPLICIT_W) {
    const R4<real> wm = v.wmesh[i];
    w[0] = wm.x; w[1] = wm.y; w[2] = wm.z;
  }
}

// the neighbour j of incidence q: the bits of the last real of its record
__device__ __forceinline__ int incidence_nbr(const HydroView<float>& v, int q) {
  return __float_as_int(__ldg(&v.igAB[2 * (size_t)q + 1].w));
}
__device__ __forceinline__ int incidence_nbr(const HydroView<double>& v, int q) {
  return (int)__double_as_longlong(__ldg(&v.igAB[2 * (size_t)q + 1].w));
}

// The limited gradient of cell i (valid) by the G lanes of its group: lane
// `lane` takes the incidences lane, lane+G, ...; the results are stored.
// ii is a valid cell index for the lanes of an invalid group (their loads
// stay in bounds; nothing is stored).  Returns the cell's record through
// Wi (rho, v) and Pi, and its geometry {1/V, s - r} through cg.
// ENT: the entropy switch is on, so the entropic function A is a sixth
// limited variable and the largest kinetic energy around the cell is kept
// for the cold-flow criterion.
// pred: also write the cell's record predicted over hdt (static mesh, lab
// frame: W - hdt A(W) grad W with the limited gradients; Sec. 3.3's
// half-step prediction, which on a static mesh does not depend on the face).
template <typename real, int G, bool ENT = false>
__device__ __forceinline__ void grad_cell(const HydroView<real>& v, int i, int ii, bool valid, int lane, R4<real>& Wi,
                                          real& Pi, R4<real>& cg, bool pred = false, real hdt = (real)0) {
  constexpr int UNR = 1;                               // incidences in flight per lane
  constexpr int NV = ENT ? 6 : 5;
  Wi = v.cw[2 * (size_t)ii];
  real phi_i[NV];
  phi_i[0] = Wi.x; phi_i[1] = Wi.y; phi_i[2] = Wi.z; phi_i[3] = Wi.w; phi_i[4] = v.cw[2 * (size_t)ii + 1].x;
  if constexpr (ENT) phi_i[5] = v.Aw[ii];
  cg = v.cgeo[ii];
  const int q0 = valid ? v.csr_off[ii] : 0;
  const int q1 = valid ? v.csr_off[ii + 1] : 0;
  real g[NV][3];
  real mx[NV], mn[NV];
#pragma unroll
  for (int a = 0; a < NV; a++) {
    g[a][0] = g[a][1] = g[a][2] = (real)0;
    mx[a] = mn[a] = phi_i[a];
  }
  // cold-flow criterion: largest 1/2 m_j |v_j - w_i|^2 over the cell and
  // its neighbours (start-of-step states)
  real wi3[3];
  real ekm = (real)0;
  const bool cold = ENT && v.alpha_s > 0.0;
  if (cold) {
    mesh_velocity(v, ii, Wi, wi3);
    const real dx = Wi.y - wi3[0], dy = Wi.z - wi3[1], dz = Wi.w - wi3[2];
    ekm = (real)0.5 * (real)v.Q[ii] * (dx * dx + dy * dy + dz * dz);
  }
  // the neighbour index of the next incidence (the last word of its record)
  // is loaded one iteration ahead, so the neighbour's state load does not
  // wait behind the record
  int jn = (q0 + lane < q1) ? incidence_nbr(v, q0 + lane) : 0;
#pragma unroll UNR
  for (int q = q0 + lane; q < q1; q += G) {
    // V grad = sum A ([phi_j - phi_i] c / r_ij + (phi_i + phi_j)/2 n_out)
    //        = sum (phi_j - phi_i) w,  w = A (c / r_ij + n_out / 2)
    // (a closed cell's sum of A n_out vanishes), w precomputed per incidence
    const int j = jn;
    if (q + G < q1) jn = incidence_nbr(v, q + G);
    R4<real> a4, b4, Wj;
    real Pj;
    if constexpr (sizeof(real) == 4) {
      // the incidence's record and the neighbour's record {W}, {P, s - r}:
      // one 32-byte load each
      ldg256(v.igAB + 2 * (size_t)q, a4, b4);
      R4<real> Pc;
      ldg256(v.cw + 2 * (size_t)j, Wj, Pc);
      Pj = Pc.x;
    } else {
      a4 = v.igAB[2 * (size_t)q];
      b4 = v.igAB[2 * (size_t)q + 1];
      Wj = v.cw[2 * (size_t)j];
      Pj = v.cw[2 * (size_t)j + 1].x;
    }
    real phi_j[NV];
    phi_j[0] = Wj.x; phi_j[1] = Wj.y; phi_j[2] = Wj.z; phi_j[3] = Wj.w; phi_j[4] = Pj;
    if constexpr (ENT) phi_j[5] = v.Aw[j];
    if (cold) {
      const real dx = Wj.y - wi3[0], dy = Wj.z - wi3[1], dz = Wj.w - wi3[2];
      const real ek = (real)0.5 * (real)v.Q[j] * (dx * dx + dy * dy + dz * dz);
      ekm = ek > ekm ? ek : ekm;
    }
#pragma unroll
    for (int a = 0; a < NV; a++) {
      const real d = phi_j[a] - phi_i[a];
      g[a][0] += d * a4.x;
      g[a][1] += d * a4.y;
      g[a][2] += d * a4.z;
      mx[a] = phi_j[a] > mx[a] ? phi_j[a] : mx[a];
      mn[a] = phi_j[a] < mn[a] ? phi_j[a] : mn[a];
    }
  }
  const real invV = cg.x;
#pragma unroll
  for (int a = 0; a < NV; a++) {
    g[a][0] = group_sum<G>(g[a][0]) * invV;
    g[a][1] = group_sum<G>(g[a][1]) * invV;
    g[a][2] = group_sum<G>(g[a][2]) * invV;
    mx[a] = group_max<G>(mx[a]);
    mn[a] = group_min<G>(mn[a]);
  }
  if (v.limit) {
    // alpha = min(1, min over incidences of psi), psi = (max - phi_i) / dphi
    // for dphi > 0 and (min - phi_i) / dphi for dphi < 0, taken branch-free
    // as 1 / max(1, max of dphi / (max - phi_i) or dphi / (min - phi_i)): the
    // two reciprocals once per cell and variable, one product per incidence.
    // (An extremal cell's reciprocal is infinite, so a dphi towards it gives
    // alpha = 0; a dphi of 0 gives NaN, which fmax ignores.)
    real bmax[NV], rmx[NV], rmn[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) {
      bmax[a] = (real)0;
      rmx[a] = (real)1 / (mx[a] - phi_i[a]);
      rmn[a] = (real)-1 / (phi_i[a] - mn[a]);
    }
  #pragma unroll UNR
  for (int q = q0 + lane; q < q1; q += G) {
      // f - s_i of the incidence
      const R4<real> b4 = v.igAB[2 * (size_t)q + 1];
      const real fx = b4.x, fy = b4.y, fz = b4.z;
#pragma unroll
      for (int a = 0; a < NV; a++) {
        const real dphi = g[a][0] * fx + g[a][1] * fy + g[a][2] * fz;
        bmax[a] = fmax(bmax[a], dphi * (dphi > (real)0 ? rmx[a] : rmn[a]));
      }
    }
#pragma unroll
    for (int a = 0; a < NV; a++) {
      const real al = (real)1 / fmax((real)1, group_max<G>(bmax[a]));
      g[a][0] *= al;
      g[a][1] *= al;
      g[a][2] *= al;
    }
  }
  if (valid) {
    R4<real> o[4];
    o[0].x = g[0][0]; o[0].y = g[0][1]; o[0].z = g[0][2]; o[0].w = g[4][0];
    o[1].x = g[1][0]; o[1].y = g[1][1]; o[1].z = g[1][2]; o[1].w = g[4][1];
    o[2].x = g[2][0]; o[2].y = g[2][1]; o[2].z = g[2][2]; o[2].w = g[4][2];
    o[3].x = g[3][0]; o[3].y = g[3][1]; o[3].z = g[3][2]; o[3].w = (real)0;
    R4<real>* go = v.grad + 4 * (size_t)i;
#pragma unroll
    for (int r = 0; r < 4; r++)
      if (r % G == lane) go[r] = o[r];
    if constexpr (ENT) {
      if (lane == 0) {
        R4<real> ga;
        ga.x = g[5][0]; ga.y = g[5][1]; ga.z = g[5][2]; ga.w = (real)0;
        v.gradA[i] = ga;
      }
    }
    if (pred && lane == 0) {
      // dW/dt = -A(W) grad W in the lab frame (the face-frame boost of a
      // static mesh is zero): d rho/dt = -(v.grad rho + rho div v),
      // dv/dt = -(v.grad) v - grad P / rho, dP/dt = -(gamma P div v + v.grad P)
      // (explicitly rounded: the persistent step kernel must round alike)
      const real rho = phi_i[0], vx = phi_i[1], vy = phi_i[2], vz = phi_i[3], P = phi_i[4];
      const real divv = rn_add(rn_add(g[1][0], g[2][1]), g[3][2]);
      const real ir = (real)1 / rho;
      const real mh = -hdt;
      R4<real> a, b;
      a.x = rn_fma(mh, rn_fma(rho, divv, rn_dot3(vx, vy, vz, g[0][0], g[0][1], g[0][2])), rho);
      a.y = rn_fma(mh, rn_fma(g[4][0], ir, rn_dot3(vx, vy, vz, g[1][0], g[1][1], g[1][2])), vx);
      a.z = rn_fma(mh, rn_fma(g[4][1], ir, rn_dot3(vx, vy, vz, g[2][0], g[2][1], g[2][2])), vy);
      a.w = rn_fma(mh, rn_fma(g[4][2], ir, rn_dot3(vx, vy, vz, g[3][0], g[3][1], g[3][2])), vz);
      b.x = rn_fma(mh, rn_fma(rn_mul(v.gas.g, P), divv, rn_dot3(vx, vy, vz, g[4][0], g[4][1], g[4][2])), P);
      b.y = cg.y; b.z = cg.z; b.w = cg.w;       // s - r
      v.cwp[2 * (size_t)i] = a;
      v.cwp[2 * (size_t)i + 1] = b;
      if constexpr (ENT) v.Apw[i] = rn_fma(mh, rn_dot3(vx, vy, vz, g[5][0], g[5][1], g[5][2]), phi_i[5]);
    }
  }
  if (cold) {
    ekm = group_max<G>(ekm);
    if (valid && lane == 0) v.ekmax[i] = ekm;
  }
  Pi = phi_i[4];
}

// Cell i's Courant time R_i / (c_i + |v_i - w_i|) (eq. EqnTiStep), from its
// record {rho, v} and pressure; with the regularity correction also its
// corrected mesh velocity of the step (written to wcorr).
template <typename real>
__device__ __forceinline__ real courant_time(const HydroView<real>& v, int i, const R4<real>& Wi, real Pi) {
  real w3[3];
  mesh_velocity(v, i, Wi, w3);
  // (explicitly rounded: the persistent step kernel must round alike)
  const real cs = xsqrt(rn_mul(v.gas.g, Pi) / Wi.x);
  const real Ri = v.crad[i];
  if (v.regularize) {
    // Sec. 4.1, eq. (EqnShapeCorrVel): towards the centre of mass at the
    // sound speed once the generator is off it by more than eta R_i
    const R4<real> cg = v.cgeo[i];
    const real sx = cg.y, sy = cg.z, sz = cg.w;   // s - r
    const real d = xsqrt(rn_dot3(sx, sy, sz, sx, sy, sz));
    const real er = rn_mul(v.eta_r, Ri);
    const real ramp = d >= rn_mul((real)1.1, er)
                          ? (real)1
                          : (d >= rn_mul((real)0.9, er) ? rn_fma((real)-0.9, er, d) / rn_mul((real)0.2, er) : (real)0);
    if (ramp > (real)0) {
      const real f = rn_mul(rn_mul(v.chi_r, cs), ramp) / d;
      w3[0] = rn_fma(f, sx, w3[0]); w3[1] = rn_fma(f, sy, w3[1]); w3[2] = rn_fma(f, sz, w3[2]);
    }
    R4<real> wc;
    wc.x = w3[0]; wc.y = w3[1]; wc.z = w3[2]; wc.w = (real)0;
    v.wcorr[i] = wc;
  }
  const real dx = Wi.y - w3[0], dy = Wi.z - w3[1], dz = Wi.w - w3[2];
  return Ri / rn_add(cs, xsqrt(rn_dot3(dx, dy, dz, dx, dy, dz)));
}

// The CTA's minimum of tc folded into box b's Courant minimum: one integer
// atomic per CTA (positive doubles order like their bit patterns; min is
// order independent, so this is exact).  Every thread of the CTA calls it.
template <typename real>
__device__ __forceinline__ void courant_block_min(const HydroView<real>& v, real tc, int b) {
  tc = group_min<32>(tc);
  __shared__ real wmin[CELL_TILE / 32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = tc;
  __syncthreads();
  if (threadIdx.x == 0) {
    real m = wmin[0];
    for (int w = 1; w < CELL_TILE / 32; w++) m = wmin[w] < m ? wmin[w] : m;
    const double md = (double)m;
    if (md > 0.0 && md < 1.0e300)
      atomicMin(v.cour_bits + b, (unsigned long long)__double_as_longlong(md));
  }
  __syncthreads();   // `wmin` is reused by the next work item of a persistent CTA
}

// work item wi: cells of tile wi (one thread per cell): the per-box Courant
// minimum of a static mesh's step, which its gradient kernel needs
template <typename real>
__device__ __forceinline__ void courant_item(const HydroView<real>& v, int wi) {
  const Tile t = v.ctiles[wi];
  const int i = t.begin + (int)threadIdx.x;
  real tc = (real)3.0e38;
  if (i < t.end) tc = courant_time(v, i, v.cw[2 * (size_t)i], v.cw[2 * (size_t)i + 1].x);
  courant_block_min(v, tc, t.box);
}

template <typename real>
__global__ void __launch_bounds__(CELL_TILE) k_courant(HydroView<real> v) {
  courant_item<real>(v, blockIdx.x);
}

// work item wi: cells of tile wi/G, sub-block wi%G (CELL_TILE threads):
// gradients and limiter.  Static mesh: also the half-step predicted records,
// over half of the box's step (courant_item ran before, so the box's Courant
// minimum is complete).  Moving mesh: also the Courant minimum, one lane per
// cell.
template <typename real, int G, bool ENT = false>
__device__ __forceinline__ void grad_item(const HydroView<real>& v, int wi) {
  constexpr int CELLS = CELL_TILE / G;                 // cells per CTA
  const Tile t = v.ctiles[wi / G];
  const int lane = (int)threadIdx.x % G;
  const int i = t.begin + (int)(wi % G) * CELLS + (int)threadIdx.x / G;
  const bool valid = i < t.end;
  const int ii = valid ? i : t.begin;
  R4<real> Wi, cg;
  real Pi;
  if (v.pred) {
    // half the box's step, by one thread (the FP64 arithmetic of box_dt runs
    // on the narrow FP64 pipe)
    __shared__ real s_hdt;
    if (threadIdx.x == 0) s_hdt = (real)(0.5 * box_dt(v, t.box));
    __syncthreads();
    const real hdt = s_hdt;
    __syncthreads();   // `s_hdt` is rewritten by the next work item of a persistent CTA
    grad_cell<real, G, ENT>(v, i, ii, valid, lane, Wi, Pi, cg, true, hdt);
  } else {
    grad_cell<real, G, ENT>(v, i, ii, valid, lane, Wi, Pi, cg);
    real tc = (real)3.0e38;
    if (valid && lane == 0) tc = courant_time(v, i, Wi, Pi);
    courant_block_min(v, tc, t.box);
  }
}

template <typename real, int G, bool ENT>
__global__ void __launch_bounds__(CELL_TILE, sizeof(real) == 4 ? 4 : 2) k_gradients(HydroView<real> v) {
  grad_item<real, G, ENT>(v, blockIdx.x);
}

// ------------------------------------------------------------ A5+A6+A7
struct FaceStats {
  int iters, guard, vacuum, fail, fallback;
};

// A cell's record as the flux computation reads it: {rho, v}, {P, s - r},
// the four gradient vectors and, with the entropy switch, A and grad A.
template <typename real>
struct CellRec {
  R4<real> W, Pc, g0, g1, g2, g3;
  real A;
  R4<real> gA;
};

template <typename real, bool ENT>
__device__ __forceinline__ CellRec<real> load_cell_rec(const HydroView<real>& v, int i) {
  CellRec<real> r;
  r.W = v.cw[2 * (size_t)i];
  r.Pc = v.cw[2 * (size_t)i + 1];
  const R4<real>* gp = v.grad + 4 * (size_t)i;
  r.g0 = gp[0];
  r.g1 = gp[1];
  r.g2 = gp[2];
  r.g3 = gp[3];
  if constexpr (ENT) {
    r.A = v.Aw[i];
    r.gA = v.gradA[i];
  }
  return r;
}

// One side of a face: boost into the face frame, spatial extrapolation to
// the face centroid and half-step prediction with A(W') at the cell centre
// (gradients are frame independent).  hsgn = +1/2 for the left cell, -1/2
// for the right one (f - s_i = hsgn |d| n + c - (s_i - r_i)).
template <typename real, bool ENT>
__device__ __forceinline__ void side_extrapolate(const GasC<real>& G, const CellRec<real>& rc, real hsgn,
                                                 const real* n, real sep, const real* c, const real* w, real hdt,
                                                 real* Wp, real* Wpp, real& Aface) {
  const R4<real>& Wi = rc.W;
  const R4<real>& cg = rc.Pc;   // {P, s - r}
  const real P = cg.x;
  const R4<real>& g0 = rc.g0;
  const R4<real>& g1 = rc.g1;
  const R4<real>& g2 = rc.g2;
  const R4<real>& g3 = rc.g3;
  // f - s_i
  const real fx = hsgn * sep * n[0] + c[0] - cg.y;
  const real fy = hsgn * sep * n[1] + c[1] - cg.z;
  const real fz = hsgn * sep * n[2] + c[2] - cg.w;
  // boost into the face frame
  const real rho = Wi.x;
  const real ux = Wi.y - w[0], uy = Wi.z - w[1], uz = Wi.w - w[2];
  Wp[0] = rho; Wp[1] = ux; Wp[2] = uy; Wp[3] = uz; Wp[4] = P;
  const real divv = g1.x + g2.y + g3.z;
  const real ir = (real)1 / rho;
  Wpp[0] = rho + (g0.x * fx + g0.y * fy + g0.z * fz) - hdt * (ux * g0.x + uy * g0.y + uz * g0.z + rho * divv);
  Wpp[1] = ux + (g1.x * fx + g1.y * fy + g1.z * fz) - hdt * (ux * g1.x + uy * g1.y + uz * g1.z + g0.w * ir);
  Wpp[2] = uy + (g2.x * fx + g2.y * fy + g2.z * fz) - hdt * (ux * g2.x + uy * g2.y + uz * g2.z + g1.w * ir);
  Wpp[3] = uz + (g3.x * fx + g3.y * fy + g3.z * fz) - hdt * (ux * g3.x + uy * g3.y + uz * g3.z + g2.w * ir);
  Wpp[4] = P + (g0.w * fx + g1.w * fy + g2.w * fz) -
           hdt * (G.g * P * divv + ux * g0.w + uy * g1.w + uz * g2.w);
  if constexpr (ENT) {
    // entropic function A (Sec. 3.5): reconstructed like the primitives and
    // advected, dA/dt = -v'.grad A; the cell value if that is not positive
    const real A = rc.A;
    const R4<real>& ga = rc.gA;
    const real Ap = A + (ga.x * fx + ga.y * fy + ga.z * fz) - hdt * (ux * ga.x + uy * ga.y + uz * ga.z);
    Aface = Ap > (real)0 ? Ap : A;
  }
}

// Per-face state between the extrapolation (face_prepare) and the Riemann
// solve + flux (face_finish); the learned form runs the proposal network
// between the two on the tensor cores.
template <typename real>
struct FaceWork {
  int k;
  bool valid;
  int2 lr;
  real n[3], A, w[3];
  real WppL[5], WppR[5];
  real uL, uR;
  real AL, AR;                 // entropic function of each side (entropy switch)
  int fallback;
};

// hdtL, hdtR: the time over which each side is predicted (half the step; with
// individual time steps, the time from the side's last activation to the
// middle of the face's step).  lr, G0, G1: the face's cells and geometry
// records; recL, recR: its cells' records (loaded by the caller).
// STATIC: the caller knows the mesh is static (w = 0), so the face-velocity
// work compiles away.
template <typename real, bool ENT, bool STATIC = false>
__device__ __forceinline__ void face_prepare_rec(const HydroView<real>& v, int k, bool valid, real hdtL, real hdtR,
                                                 int2 lr, const R4<real>& G0, const R4<real>& G1,
                                                 const CellRec<real>& recL, const CellRec<real>& recR,
                                                 FaceWork<real>& f) {
  f.k = k;
  f.valid = valid;
  f.lr = lr;
  const real n[3] = {G0.x, G0.y, G0.z};
  const real sep = G0.w;
  const real c[3] = {G1.x, G1.y, G1.z};
  f.A = G1.w;
  // face velocity: mean of the generators' velocities plus the normal motion
  // of the face centroid from their relative motion about the midpoint
  real w[3] = {(real)0, (real)0, (real)0};
  if (!STATIC && v.mode != AMM_EULERIAN) {
    real wl[3], wr[3];
    if (v.regularize) {
      // the generators' velocities with the regularity correction, from the
      // gradient kernel
      const R4<real> a = v.wcorr[lr.x], b = v.wcorr[lr.y];
      wl[0] = a.x; wl[1] = a.y; wl[2] = a.z;
      wr[0] = b.x; wr[1] = b.y; wr[2] = b.z;
    } else if (v.mode == AMM_LAGRANGIAN) {
      wl[0] = recL.W.y; wl[1] = recL.W.z; wl[2] = recL.W.w;
      wr[0] = recR.W.y; wr[1] = recR.W.z; wr[2] = recR.W.w;
    } else {
      const R4<real> a = v.wmesh[lr.x], b = v.wmesh[lr.y];
      wl[0] = a.x; wl[1] = a.y; wl[2] = a.z;
      wr[0] = b.x; wr[1] = b.y; wr[2] = b.z;
    }
    const real rot = ((wl[0] - wr[0]) * c[0] + (wl[1] - wr[1]) * c[1] + (wl[2] - wr[2]) * c[2]) / sep;
#pragma unroll
    for (int d = 0; d < 3; d++) w[d] = (real)0.5 * (wl[d] + wr[d]) + rot * n[d];
  }
  real WpL[5], WpR[5];
  f.AL = f.AR = (real)0;
  side_extrapolate<real, ENT>(v.gas, recL, (real)0.5, n, sep, c, w, hdtL, WpL, f.WppL, f.AL);
  side_extrapolate<real, ENT>(v.gas, recR, (real)-0.5, n, sep, c, w, hdtR, WpR, f.WppR, f.AR);
  f.fallback = 0;
  if (!(f.WppL[0] > (real)0) || !(f.WppL[4] > (real)0) || !(f.WppR[0] > (real)0) || !(f.WppR[4] > (real)0)) {
#pragma unroll
    for (int a = 0; a < 5; a++) {
      f.WppL[a] = WpL[a];
      f.WppR[a] = WpR[a];
    }
    if constexpr (ENT) {
      f.AL = recL.A;
      f.AR = recR.A;
    }
    f.fallback = 1;
  }
  // rotate: normal component and transverse vector
  f.uL = f.WppL[1] * n[0] + f.WppL[2] * n[1] + f.WppL[3] * n[2];
  f.uR = f.WppR[1] * n[0] + f.WppR[2] * n[1] + f.WppR[3] * n[2];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    f.n[d] = n[d];
    f.w[d] = w[d];
  }
  if (v.harvest && valid) {
    float* h = v.harvest + 6 * (size_t)k;
    h[0] = (float)f.WppL[0]; h[1] = (float)f.uL; h[2] = (float)f.WppL[4];
    h[3] = (float)f.WppR[0]; h[4] = (float)f.uR; h[5] = (float)f.WppR[4];
  }
}

// the same with every record read from global memory
template <typename real, bool ENT>
__device__ __forceinline__ void face_prepare(const HydroView<real>& v, int k, bool valid, real hdtL, real hdtR,
                                             FaceWork<real>& f) {
  const int2 lr = v.lr[k];
  const R4<real> G0 = v.fgeo[2 * (size_t)k];
  const R4<real> G1 = v.fgeo[2 * (size_t)k + 1];
  const CellRec<real> recL = load_cell_rec<real, ENT>(v, lr.x);
  const CellRec<real> recR = load_cell_rec<real, ENT>(v, lr.y);
  face_prepare_rec<real, ENT>(v, k, valid, hdtL, hdtR, lr, G0, G1, recL, recR, f);
}

// Static mesh: a side's face state from its cell's predicted record (the
// gradient kernel's W - hdt A(W) grad W; with w = 0 the face frame is the lab
// frame, so the prediction does not depend on the face), extrapolated to the
// face centroid: W_p + grad W . (f - s_i).  Equal in exact arithmetic to
// side_extrapolate with w = 0.  A_raw: the cell's entropic function, taken
// where the extrapolated one is not positive.
template <typename real, bool ENT>
__device__ __forceinline__ void side_from_pred(const CellRec<real>& rp, real A_raw, real hsgn, const real* n, real sep,
                                               const real* c, real* Wpp, real& Aface) {
  const R4<real>& Wq = rp.W;    // predicted {rho, v}
  const R4<real>& cg = rp.Pc;   // {predicted P, s - r}
  const R4<real>& g0 = rp.g0;
  const R4<real>& g1 = rp.g1;
  const R4<real>& g2 = rp.g2;
  const R4<real>& g3 = rp.g3;
  // (explicitly rounded: the persistent step kernel must round alike)
  const real hs = rn_mul(hsgn, sep);
  const real fx = rn_add(rn_fma(hs, n[0], c[0]), -cg.y);
  const real fy = rn_add(rn_fma(hs, n[1], c[1]), -cg.z);
  const real fz = rn_add(rn_fma(hs, n[2], c[2]), -cg.w);
  Wpp[0] = rn_add(Wq.x, rn_dot3(g0.x, g0.y, g0.z, fx, fy, fz));
  Wpp[1] = rn_add(Wq.y, rn_dot3(g1.x, g1.y, g1.z, fx, fy, fz));
  Wpp[2] = rn_add(Wq.z, rn_dot3(g2.x, g2.y, g2.z, fx, fy, fz));
  Wpp[3] = rn_add(Wq.w, rn_dot3(g3.x, g3.y, g3.z, fx, fy, fz));
  Wpp[4] = rn_add(cg.x, rn_dot3(g0.w, g1.w, g2.w, fx, fy, fz));
  if constexpr (ENT) {
    const R4<real>& ga = rp.gA;
    const real Ap = rn_add(rp.A, rn_dot3(ga.x, ga.y, ga.z, fx, fy, fz));
    Aface = Ap > (real)0 ? Ap : A_raw;
  }
}

// face_prepare_rec for a static mesh from the cells' predicted records
// (pL, pR; their A is the predicted entropic function, AL_raw / AR_raw the
// cells' own).  A face whose extrapolated state is not positive falls back
// to the cells' current states (read here, from cw).
template <typename real, bool ENT>
__device__ __forceinline__ void face_prepare_pred(const HydroView<real>& v, int k, bool valid, int2 lr,
                                                  const R4<real>& G0, const R4<real>& G1, const CellRec<real>& pL,
                                                  const CellRec<real>& pR, real AL_raw, real AR_raw,
                                                  FaceWork<real>& f) {
  f.k = k;
  f.valid = valid;
  f.lr = lr;
  const real n[3] = {G0.x, G0.y, G0.z};
  const real sep = G0.w;
  const real c[3] = {G1.x, G1.y, G1.z};
  f.A = G1.w;
  f.AL = f.AR = (real)0;
  side_from_pred<real, ENT>(pL, AL_raw, (real)0.5, n, sep, c, f.WppL, f.AL);
  side_from_pred<real, ENT>(pR, AR_raw, (real)-0.5, n, sep, c, f.WppR, f.AR);
  f.fallback = 0;
  if (!(f.WppL[0] > (real)0) || !(f.WppL[4] > (real)0) || !(f.WppR[0] > (real)0) || !(f.WppR[4] > (real)0)) {
    const R4<real> WL = v.cw[2 * (size_t)lr.x], PL = v.cw[2 * (size_t)lr.x + 1];
    const R4<real> WR = v.cw[2 * (size_t)lr.y], PR = v.cw[2 * (size_t)lr.y + 1];
    f.WppL[0] = WL.x; f.WppL[1] = WL.y; f.WppL[2] = WL.z; f.WppL[3] = WL.w; f.WppL[4] = PL.x;
    f.WppR[0] = WR.x; f.WppR[1] = WR.y; f.WppR[2] = WR.z; f.WppR[3] = WR.w; f.WppR[4] = PR.x;
    if constexpr (ENT) {
      f.AL = AL_raw;
      f.AR = AR_raw;
    }
    f.fallback = 1;
  }
  f.uL = rn_dot3(f.WppL[1], f.WppL[2], f.WppL[3], n[0], n[1], n[2]);
  f.uR = rn_dot3(f.WppR[1], f.WppR[2], f.WppR[3], n[0], n[1], n[2]);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    f.n[d] = n[d];
    f.w[d] = (real)0;
  }
  if (v.harvest && valid) {
    float* h = v.harvest + 6 * (size_t)k;
    h[0] = (float)f.WppL[0]; h[1] = (float)f.uL; h[2] = (float)f.WppL[4];
    h[3] = (float)f.WppR[0]; h[4] = (float)f.uR; h[5] = (float)f.WppR[4];
  }
}

// a cell's predicted record from global memory (static mesh)
template <typename real, bool ENT>
__device__ __forceinline__ CellRec<real> load_pred_rec(const HydroView<real>& v, int i) {
  CellRec<real> r;
  r.W = v.cwp[2 * (size_t)i];
  r.Pc = v.cwp[2 * (size_t)i + 1];
  const R4<real>* gp = v.grad + 4 * (size_t)i;
  r.g0 = gp[0];
  r.g1 = gp[1];
  r.g2 = gp[2];
  r.g3 = gp[3];
  if constexpr (ENT) {
    r.A = v.Apw[i];
    r.gA = v.gradA[i];
  }
  return r;
}

// A face of a step (hdt: half the box's step): from the predicted records on
// a static mesh, else with the face-frame prediction of face_prepare.
template <typename real, bool ENT>
__device__ __forceinline__ void face_prepare_step(const HydroView<real>& v, int k, bool valid, real hdt,
                                                  FaceWork<real>& f) {
  if (v.pred) {
    const int2 lr = v.lr[k];
    const R4<real> G0 = v.fgeo[2 * (size_t)k];
    const R4<real> G1 = v.fgeo[2 * (size_t)k + 1];
    const CellRec<real> pL = load_pred_rec<real, ENT>(v, lr.x);
    const CellRec<real> pR = load_pred_rec<real, ENT>(v, lr.y);
    real AL = (real)0, AR = (real)0;
    if constexpr (ENT) {
      AL = v.Aw[lr.x];
      AR = v.Aw[lr.y];
    }
    face_prepare_pred<real, ENT>(v, k, valid, lr, G0, G1, pL, pR, AL, AR, f);
  } else {
    face_prepare<real, ENT>(v, k, valid, hdt, hdt, f);
  }
}

// What one face contributes to the step's reductions: the magnitudes of its
// A F components as float bits (non-negative floats order like their bits),
// its Newton iterations and flags.
struct FaceOut {
  unsigned m[6];
  unsigned iters;
  bool guard, vacuum, fail, fallback;
};

// Riemann solve, flux of the moving face and its stores (valid faces only);
// the face's contributions to the reductions in `o` (zero for an invalid
// face).  have_guess: start Newton from `guess` in place of the two-shock
// estimate.  pre: the caller has the sides' sound speeds and the linearised
// star pressure (cs = {c_L, c_R, p_pv}) already.
template <typename real, bool ENT>
__device__ __forceinline__ void face_finish_core(const HydroView<real>& v, const FaceWork<real>& f, bool have_guess,
                                                 real guess, FaceOut& o, bool pre = false, const real* cs = nullptr) {
  const GasC<real>& G = v.gas;
  const bool valid = f.valid;
  real rhoF, uF, pF, ps;
  RiemannInfo info;
  const int side =
      pre ? riemann_sample_c(f.WppL[0], f.uL, f.WppL[4], f.WppR[0], f.uR, f.WppR[4], cs[0], cs[1], cs[2], G, v.tol,
                             v.tol_r, v.maxit, have_guess, guess, rhoF, uF, pF, info, ps)
          : riemann_sample(f.WppL[0], f.uL, f.WppL[4], f.WppR[0], f.uR, f.WppR[4], G, v.tol, v.tol_r, v.maxit,
                           have_guess, guess, rhoF, uF, pF, info, ps);
  const real* Wt = side ? f.WppR : f.WppL;
  const real ut = side ? f.uR : f.uL;
  real vlab[3];
#pragma unroll
  for (int d = 0; d < 3; d++) vlab[d] = uF * f.n[d] + (Wt[1 + d] - ut * f.n[d]) + f.w[d];
  const real v2 = vlab[0] * vlab[0] + vlab[1] * vlab[1] + vlab[2] * vlab[2];
  const real vn = vlab[0] * f.n[0] + vlab[1] * f.n[1] + vlab[2] * f.n[2];
  const real mflux = rhoF * uF;
  const real A = f.A;
  R4<real> fout;
  fout.x = A * mflux;
  fout.y = A * (mflux * vlab[0] + pF * f.n[0]);
  fout.z = A * (mflux * vlab[1] + pF * f.n[1]);
  fout.w = A * (mflux * vlab[2] + pF * f.n[2]);
  const real fE = A * (((real)0.5 * rhoF * v2 + pF * G.inv_gm1) * uF + pF * vn);
  if (valid) {
    v.flux[f.k] = fout;
    v.fluxE[f.k] = fE;
  }
  real fS = (real)0;
  if constexpr (ENT) {
    // Sec. 3.5: entropy flux rho_F u_F A_U (A_U of the upwind side by the
    // sign of u_F) and the largest Mach number of the problem's shocks (the
    // waves with p* above the pressure ahead of them)
    fS = A * (rhoF * uF) * (uF > (real)0 ? f.AL : f.AR);
    real mach = (real)1;
    if (!info.vacuum) {
      if (ps > f.WppL[4]) mach = xsqrt((real)1 + G.shock_a * (ps / f.WppL[4] - (real)1));
      if (ps > f.WppR[4]) {
        const real mr = xsqrt((real)1 + G.shock_a * (ps / f.WppR[4] - (real)1));
        mach = mr > mach ? mr : mach;
      }
    }
    if (valid) {
      v.fluxS[f.k] = fS;
      v.machf[f.k] = mach;
    }
  }
#pragma unroll
  for (int a = 0; a < 6; a++) o.m[a] = 0u;
  if (valid) {
    o.m[0] = __float_as_uint(fabsf((float)fout.x));
    o.m[1] = __float_as_uint(fabsf((float)fout.y));
    o.m[2] = __float_as_uint(fabsf((float)fout.z));
    o.m[3] = __float_as_uint(fabsf((float)fout.w));
    o.m[4] = __float_as_uint(fabsf((float)fE));
    if constexpr (ENT) o.m[5] = __float_as_uint(fabsf((float)fS));
  }
  o.iters = valid ? (unsigned)info.iters : 0u;
  o.guard = valid && info.guard;
  o.vacuum = valid && info.vacuum;
  o.fail = valid && info.fail;
  o.fallback = valid && f.fallback;
}

// Adds a warp's statistics to the device totals (lane 0 of a full warp
// calls it with warp-reduced values).
__device__ __forceinline__ void stats_add(DeviceStats* S, unsigned* box_status, int box, unsigned long long faces,
                                          unsigned long long iters, unsigned guard, unsigned vacuum, unsigned fail,
                                          unsigned fallback, unsigned maxit) {
  if (faces) atomicAdd(&S->faces, faces);
  if (iters) atomicAdd(&S->newton_iters, iters);
  if (guard) atomicAdd(&S->guard, (unsigned long long)guard);
  if (vacuum) atomicAdd(&S->vacuum, (unsigned long long)vacuum);
  if (fallback) atomicAdd(&S->fallback, (unsigned long long)fallback);
  if (fail) {
    atomicAdd(&S->newton_fail, (unsigned long long)fail);
    atomicOr(&S->status, (unsigned)ST_NEWTON_CAP);
    if (box >= 0) atomicOr(box_status + box, (unsigned)ST_NEWTON_CAP);
  }
  if (maxit) atomicMax(&S->newton_max, maxit);
}

// Riemann solve, flux of the moving face, stores, and the CTA's reductions
// (largest |A F| per component, Newton statistics).  All B threads call it.
template <typename real, int B, bool ENT>
__device__ __forceinline__ void face_finish(const HydroView<real>& v, const FaceWork<real>& f, int box, int nf_here,
                                            bool have_guess, real guess) {
  const bool valid = f.valid;
  FaceOut o;
  face_finish_core<real, ENT>(v, f, have_guess, guess, o);
  if (sizeof(real) == 4 && v.fixed_acc) {
    // largest |A F| per component for the exact fixed-point sums
    constexpr int NM = ENT ? 6 : 5;
    __shared__ unsigned wm[B / 32][NM];
#pragma unroll
    for (int a = 0; a < NM; a++) {
      const unsigned r = __reduce_max_sync(0xffffffffu, o.m[a]);
      if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5][a] = r;
    }
    __syncthreads();
    if (threadIdx.x < NM) {
      unsigned r = 0u;
      for (int w = 0; w < B / 32; w++) r = wm[w][threadIdx.x] > r ? wm[w][threadIdx.x] : r;
      atomicMax(v.fmax_bits + FMAX_STRIDE * box + threadIdx.x, r);
    }
  }
  // statistics: warp reductions (no contended shared-memory atomics), one
  // slot per warp in shared memory, then a few global atomics per CTA
  const unsigned full = 0xffffffffu;
  const unsigned it = o.iters;
  unsigned mine[6];
  mine[0] = __reduce_add_sync(full, it);
  mine[1] = __popc(__ballot_sync(full, o.guard));
  mine[2] = __popc(__ballot_sync(full, o.vacuum));
  mine[3] = __popc(__ballot_sync(full, o.fail));
  mine[4] = __popc(__ballot_sync(full, o.fallback));
  mine[5] = __reduce_max_sync(full, it);
  __shared__ unsigned sh[B / 32][22];
  const int wid = (int)threadIdx.x >> 5, ln = (int)threadIdx.x & 31;
  // the iteration histogram: the lanes with equal counts by one match, the
  // lowest of them writes their number (distinct bins; absent bins stay 0)
  if (ln < 16) sh[wid][ln] = 0u;
  __syncwarp();
  {
    const unsigned key = valid ? (it < 15u ? it : 15u) : 0xffffffffu;
    const unsigned m = __match_any_sync(full, key);
    if (valid && ln == __ffs(m) - 1) sh[wid][key] = __popc(m);
  }
  if (ln == 0) {
#pragma unroll
    for (int s = 0; s < 6; s++) sh[wid][16 + s] = mine[s];
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    unsigned tot = 0;
    for (int w = 0; w < B / 32; w++) tot += sh[w][threadIdx.x];
    if (tot) atomicAdd(&v.stats->hist[threadIdx.x], (unsigned long long)tot);
  } else if (threadIdx.x == 16) {
    unsigned t[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < B / 32; w++) {
      for (int s = 0; s < 5; s++) t[s] += sh[w][16 + s];
      t[5] = sh[w][21] > t[5] ? sh[w][21] : t[5];
    }
    stats_add(v.stats, v.box_status, box, (unsigned long long)(nf_here > 0 ? nf_here : 0), t[0], t[1], t[2], t[3],
              t[4], t[5]);
  }
}

// B threads (faces) per CTA; a tile of FACE_TILE faces spans FACE_TILE/B CTAs
template <typename real, int B, bool ENT>
__device__ __forceinline__ void flux_item(const HydroView<real>& v, int wi) {
  constexpr int SUB = FACE_TILE / B;
  const Tile t = v.ftiles[wi / SUB];
  const int first = t.begin + (int)(wi % SUB) * B;
  const int k0 = first + (int)threadIdx.x;
  const bool valid = k0 < t.end;
  __shared__ real s_hdt;
  if (threadIdx.x == 0) s_hdt = (real)(0.5 * box_dt(v, t.box));
  __syncthreads();
  FaceWork<real> f;
  face_prepare_step<real, ENT>(v, valid ? k0 : t.begin, valid, s_hdt, f);
  face_finish<real, B, ENT>(v, f, t.box, min(B, t.end - first), false, (real)0);
}

template <typename real, int B, bool ENT>
__global__ void __launch_bounds__(B, sizeof(real) == 4 ? 4 * FACE_TILE / B : FACE_TILE / B) k_flux(HydroView<real> v) {
  flux_item<real, B, ENT>(v, blockIdx.x);
}

// ------------------------------------------------------------ A8+A1+A9
// Fixed-point image of an FP32 value: x * 2^s as an int64, truncated toward
// zero, with s = 188 - headroom - eb and eb the biased exponent of the largest
// magnitude of the component, so every |x| 2^s < 2^(62 - headroom) and a sum
// over at most 2^headroom terms cannot overflow; the image is added to `acc`
// with the sign of x flipped when `flip` is set (the incidence's side).
// Built from the float's bits on the integer pipe (a float-to-int64
// conversion instruction would run on GB300's narrow FP64 pipe): with the
// 24-bit significand M and biased exponent e <= eb, the image is
// floor(M 2^(e - eb + 38 - headroom)) = (M 2^38) >> (eb + headroom - e), one
// right shift.  Zero (e = 0; denormals are flushed in the FP32 form) adds 0;
// Inf/NaN sets `bad`.  ebh = eb + headroom.
__device__ __forceinline__ void add_fixed(long long& acc, float x, int ebh, bool flip, bool& bad) {
  const unsigned u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xffu);
  bad |= (e == 255);
  const unsigned long long M = (e != 0) ? (unsigned long long)((u & 0x7fffffu) | 0x800000u) : 0ull;
  const long long X = (long long)((M << 38) >> min((unsigned)(ebh - e), 63u));
  const long long neg = -(long long)(((u >> 31) ^ (unsigned)flip) & 1u);   // 0 or all ones
  acc += (X ^ neg) - neg;
}

// 2^(eb - 188 + headroom) in FP64 (exact)
__device__ __forceinline__ double fixed_scale(int eb, int headroom) {
  return __longlong_as_double((long long)(1023 + eb - 188 + headroom) << 52);
}

// rho^gamma in the bulk precision (the FP32 forms' entropy switch takes it
// in FP32, like the rest of their bulk arithmetic)
template <typename real>
__device__ __forceinline__ double rho_pow_gamma(const HydroView<real>& v, double rho) {
  if constexpr (sizeof(real) == 8) {
    return pow(rho, v.gamma);
  } else {
    return (double)xpow((float)rho, v.gas.g);
  }
}

// G consecutive lanes share a cell (as in the gradient kernel); lane l sums
// the cell's incidences l, l+G, ...; the lane partial sums are combined with
// shuffles and lane 0 applies the update.  ENT: the entropy switch of
// Sec. 3.5 (a sixth flux component, the entropy, and the per-cell choice
// between the advected entropy and the energy update).
template <typename real, int G, bool ENT = false>
__device__ __forceinline__ void update_item(const HydroView<real>& v, int wi) {
  constexpr int CELLS = CELL_TILE / G;
  constexpr int NA = ENT ? 6 : 5;
  const Tile t = v.ctiles[wi / G];
  const int lane = (int)threadIdx.x % G;
  const int i = t.begin + (int)(wi % G) * CELLS + (int)threadIdx.x / G;
  const bool valid = i < t.end;
  const int q0 = valid ? v.csr_off[i] : 0;
  const int q1 = valid ? v.csr_off[i + 1] : 0;
  const size_t n = (size_t)v.n;
  double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double d[NA];
  real mach = (real)1;
  bool bad = false;
  // per tile (one box): the fixed-point exponents and dt times the scale of
  // each component's sums, so a cell's update is one FMA per component
  __shared__ int s_eb[6];
  __shared__ double s_dts[6];
  if (threadIdx.x == 0) {
    const double dt = box_dt(v, t.box);
    for (int a = 0; a < NA; a++) {
      const int eb = (int)((v.fmax_bits[FMAX_STRIDE * t.box + a] >> 23) & 0xffu);
      s_eb[a] = eb;
      s_dts[a] = (sizeof(real) == 4 && v.fixed_acc) ? dt * fixed_scale(eb, v.headroom) : dt;
    }
  }
  __syncthreads();
  if (sizeof(real) == 4 && v.fixed_acc) {
    // Exact sums: every face flux is converted once to an int64 multiple of
    // 2^-s (s per box and component, from the step's largest |A F|) and the
    // integers are added; both cells of a face add the identical integer
    // with opposite signs, so the update conserves exactly and does not
    // depend on the summation order.  One rounding per cell remains, when
    // the integer total is scaled back to FP64.
    int ebh[NA];
#pragma unroll
    for (int a = 0; a < NA; a++) ebh[a] = s_eb[a] + v.headroom;
    long long acc[NA];
#pragma unroll
    for (int a = 0; a < NA; a++) acc[a] = 0;
#pragma unroll 4
    for (int e = q0 + lane; e < q1; e += G) {
      const int2 r = v.csr[e];
      const int k = r.x >> 1;
      const R4<real> f = v.flux[k];
      float fv[NA];
      fv[0] = (float)f.x; fv[1] = (float)f.y; fv[2] = (float)f.z; fv[3] = (float)f.w; fv[4] = (float)v.fluxE[k];
      if constexpr (ENT) {
        fv[5] = (float)v.fluxS[k];
        const real mf = v.machf[k];
        mach = mf > mach ? mf : mach;
      }
#pragma unroll
      for (int a = 0; a < NA; a++) add_fixed(acc[a], fv[a], ebh[a], (r.x & 1) != 0, bad);
    }
#pragma unroll
    for (int a = 0; a < NA; a++) acc[a] = group_sum<G>(acc[a]);
    bad = group_max<G>((int)bad) != 0;
    if (lane == 0) {
#pragma unroll
      for (int a = 0; a < NA; a++) d[a] = __ll2double_rn(acc[a]);
    }
  } else {
    double acc[NA];
#pragma unroll
    for (int a = 0; a < NA; a++) acc[a] = 0.0;
#pragma unroll 4
    for (int e = q0 + lane; e < q1; e += G) {
      const int2 r = v.csr[e];
      const int k = r.x >> 1;
      const R4<real> f = v.flux[k];
      double fv[NA];
      fv[0] = (double)f.x; fv[1] = (double)f.y; fv[2] = (double)f.z; fv[3] = (double)f.w;
      fv[4] = (double)v.fluxE[k];
      if constexpr (ENT) {
        fv[5] = (double)v.fluxS[k];
        const real mf = v.machf[k];
        mach = mf > mach ? mf : mach;
      }
#pragma unroll
      for (int a = 0; a < NA; a++) {
        if (r.x & 1)
          acc[a] -= fv[a];
        else
          acc[a] += fv[a];
      }
    }
#pragma unroll
    for (int a = 0; a < NA; a++) d[a] = group_sum<G>(acc[a]);
  }
  if constexpr (ENT) mach = group_max<G>(mach);
  unsigned nonpos = 0, keep = 0;
  if (valid && lane == 0) {
#pragma unroll
    for (int a = 0; a < 5; a++)
      q[a] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v.Q[a * n + i] - s_dts[a] * d[a];
    if constexpr (ENT) {
      // Sec. 3.5: keep the advected entropy where no shock above the
      // threshold Mach number touches the cell, or where the new thermal
      // energy is below alpha_s times the largest kinetic energy around it;
      // then P = (S/M) rho^gamma sets the thermal energy.  Otherwise the
      // energy update stands and S is re-initialised from it.
      const double Sadv = v.S[i] - s_dts[5] * d[5];
      const double m = q[0];
      const double V = v.cgeo64[i].x;
      const double rho = m / V;
      const double kin = 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / m;
      keep = ((double)mach < v.mach_thresh) ? 1u : 0u;
      if (!keep && v.alpha_s > 0.0) keep = (q[4] - kin < v.alpha_s * (double)v.ekmax[i]) ? 1u : 0u;
      double Snew;
      if (keep) {
        const double Pk = (Sadv / m) * rho_pow_gamma(v, rho);
        q[4] = kin + Pk * V / (v.gamma - 1.0);
        Snew = Sadv;
      } else {
        const double Pe = (v.gamma - 1.0) * (q[4] - kin) / V;
        Snew = m * Pe / rho_pow_gamma(v, rho);
      }
      v.S[i] = Snew;
      v.kept[i] = (unsigned char)keep;
      v.Aw[i] = (real)(Snew / m);
    }
#pragma unroll
    for (int a = 0; a < 5; a++) v.Q[a * n + i] = q[a];
    const real P = prims_from_Q(v, i, q[0], q[1], q[2], q[3], q[4]);
    nonpos = (!(q[0] > 0.0) || !(P > (real)0)) ? 1u : 0u;
  }
  // per-block FP64 sums in a fixed order (bit reproducible).  Within a warp,
  // a butterfly that halves the components each lane carries at each of the
  // first three levels (5 components padded to 8): 9 FP64 adds per lane, where
  // a shuffle tree per component takes 25 on GB300's narrow FP64 pipe.  Lane
  // 4c then holds the warp's sum of component c; the warps' sums are added in
  // warp order.
  __shared__ double red[CELL_TILE / 32][5];
  {
    const int l = (int)threadIdx.x & 31;
    const bool b4 = (l & 16) != 0, b3 = (l & 8) != 0, b2 = (l & 4) != 0;
    double w4[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const double lo = q[j], hi = (j == 0) ? q[4] : 0.0;   // components j and 4 + j
      w4[j] = (b4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b4 ? lo : hi, 16);
    }
    double w2[2];
#pragma unroll
    for (int j = 0; j < 2; j++)
      w2[j] = (b3 ? w4[2 + j] : w4[j]) + __shfl_xor_sync(0xffffffffu, b3 ? w4[j] : w4[2 + j], 8);
    double w1 = (b2 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? w2[0] : w2[1], 4);
    w1 += __shfl_xor_sync(0xffffffffu, w1, 2);
    w1 += __shfl_xor_sync(0xffffffffu, w1, 1);
    const int c = l >> 2;   // 4 b4 + 2 b3 + b2
    if ((l & 3) == 0 && c < 5) red[threadIdx.x >> 5][c] = w1;
  }
  const unsigned nbad = __syncthreads_count(nonpos);
  if constexpr (ENT) {
    const unsigned nkeep = __syncthreads_count(keep);
    if (threadIdx.x == 0 && nkeep) atomicAdd(&v.stats->kept, (unsigned long long)nkeep);
  }
  if (threadIdx.x < 5) {
    double s = red[0][threadIdx.x];
    for (int w = 1; w < CELL_TILE / 32; w++) s += red[w][threadIdx.x];
    v.partial[5 * (size_t)wi + threadIdx.x] = s;
  }
  if (threadIdx.x == 0 && nbad) {
    atomicAdd(&v.stats->nonpos, (unsigned long long)nbad);
    atomicOr(&v.stats->status, (unsigned)ST_NONPOS);
    atomicOr(v.box_status + t.box, (unsigned)ST_NONPOS);
  }
  __syncthreads();   // `red` is reused by the next work item of a persistent CTA
}

template <typename real, int G, bool ENT>
__global__ void __launch_bounds__(CELL_TILE) k_update(HydroView<real> v) {
  update_item<real, G, ENT>(v, blockIdx.x);
}

// per-tile sums of the current Q (used when no step has produced them)
template <typename real>
__global__ void __launch_bounds__(CELL_TILE) k_partial_sums(HydroView<real> v) {
  const Tile t = v.ctiles[blockIdx.x];
  const int i = t.begin + (int)threadIdx.x;
  __shared__ double red[5][CELL_TILE];
  const size_t n = (size_t)v.n;
#pragma unroll
  for (int a = 0; a < 5; a++) red[a][threadIdx.x] = (i < t.end) ? v.Q[a * n + i] : 0.0;
  __syncthreads();
  for (int s = CELL_TILE / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int a = 0; a < 5; a++) red[a][threadIdx.x] += red[a][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) {
    const size_t base = 5 * (size_t)blockIdx.x * v.update_lanes;
    v.partial[base + threadIdx.x] = red[threadIdx.x][0];
    for (int g = 1; g < v.update_lanes; g++) v.partial[base + 5 * g + threadIdx.x] = 0.0;
  }
}

// one CTA per box: ordered sum of the box's block partials; time step record
constexpr int FINISH_THREADS = 512;
template <typename real, int NT>
__device__ __forceinline__ void finish_item(const HydroView<real>& v, int b, int count_step) {
  const int t0 = v.box_first_ctile[b] * v.update_lanes, t1 = v.box_first_ctile[b + 1] * v.update_lanes;
  __shared__ double red[5][NT];
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int tt = t0 + (int)threadIdx.x; tt < t1; tt += NT)
#pragma unroll
    for (int a = 0; a < 5; a++) s[a] += v.partial[5 * (size_t)tt + a];
#pragma unroll
  for (int a = 0; a < 5; a++) red[a][threadIdx.x] = s[a];
  __syncthreads();
  for (int st = NT / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
#pragma unroll
      for (int a = 0; a < 5; a++) red[a][threadIdx.x] += red[a][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) v.totals[5 * b + threadIdx.x] = red[threadIdx.x][0];
  if (threadIdx.x == 0 && count_step) {
    v.dt_used[b] = box_dt(v, b);
    if (b == 0) atomicAdd(&v.stats->steps, 1ull);
  }
  __syncthreads();   // `red` is reused when one CTA finishes several boxes
}

template <typename real>
__global__ void k_finish(HydroView<real> v, int count_step) {
  finish_item<real, FINISH_THREADS>(v, blockIdx.x, count_step);
}

// ------------------------------------------------------------ layout moves
template <typename real>
__global__ void k_set_state(HydroView<real> v, const double* Qa, int dim, unsigned long long* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int nv = dim + 2;
  const double* q = Qa + (size_t)v.cell_perm[i] * nv;
  const double m = q[0];
  const double px = q[1], py = q[2], pz = (dim == 3) ? q[3] : 0.0;
  const double E = q[dim + 1];
  const size_t n = (size_t)v.n;
  v.Q[i] = m;
  v.Q[n + i] = px;
  v.Q[2 * n + i] = py;
  v.Q[3 * n + i] = pz;
  v.Q[4 * n + i] = E;
  const real P = prims_from_Q(v, i, m, px, py, pz, E);
  if (v.entropy) {
    // S = M P / rho^gamma from the new state, in FP64
    const double V = v.cgeo64[i].x;
    const double rho = m / V;
    const double P64 = (v.gamma - 1.0) * (E - 0.5 * (px * px + py * py + pz * pz) / m) / V;
    const double S = m * P64 / pow(rho, v.gamma);
    v.S[i] = S;
    v.Aw[i] = (real)(S / m);
    v.kept[i] = 0;
  }
  if (!(m > 0.0) || !(P > (real)0)) atomicAdd(bad, 1ull);
}

template <typename real>
__global__ void k_get_state(HydroView<real> v, double* Qa, int dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int nv = dim + 2;
  const size_t n = (size_t)v.n;
  double* q = Qa + (size_t)v.cell_perm[i] * nv;
  q[0] = v.Q[i];
  q[1] = v.Q[n + i];
  q[2] = v.Q[2 * n + i];
  if (dim == 3) q[3] = v.Q[3 * n + i];
  q[dim + 1] = v.Q[4 * n + i];
}

template <typename real>
__global__ void k_get_prims(HydroView<real> v, double* Wa, int dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int nv = dim + 2;
  const R4<real> w = v.cw[2 * (size_t)i];
  double* o = Wa + (size_t)v.cell_perm[i] * nv;
  o[0] = w.x;
  o[1] = w.y;
  o[2] = w.z;
  if (dim == 3) o[3] = w.w;
  o[dim + 1] = v.cw[2 * (size_t)i + 1].x;
}

template <typename real>
__global__ void k_get_grads(HydroView<real> v, double* ga, int dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const R4<real>* gp = v.grad + 4 * (size_t)i;
  const R4<real> g0 = gp[0], g1 = gp[1], g2 = gp[2], g3 = gp[3];
  const double gg[5][3] = {{g0.x, g0.y, g0.z}, {g1.x, g1.y, g1.z}, {g2.x, g2.y, g2.z},
                           {g3.x, g3.y, g3.z}, {g0.w, g1.w, g2.w}};
  // variables in output order rho, v_1..v_dim, P
  const int var_of[5] = {0, 1, 2, 3, 4};
  double* o = ga + (size_t)v.cell_perm[i] * (dim + 2) * dim;
  int out = 0;
  for (int a = 0; a < 5; a++) {
    if (dim == 2 && a == 3) continue;
    for (int d = 0; d < dim; d++) o[out * dim + d] = gg[var_of[a]][d];
    out++;
  }
}

template <typename real>
__global__ void k_get_flux(HydroView<real> v, double* Fa, int dim) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= v.nf) return;
  const R4<real> f = v.flux[k];
  double* o = Fa + (size_t)v.face_perm[k] * (dim + 2);
  o[0] = f.x;
  o[1] = f.y;
  o[2] = f.z;
  if (dim == 3) o[3] = f.w;
  o[dim + 1] = v.fluxE[k];
}

template <typename real>
__global__ void k_set_wmesh(HydroView<real> v, const double* wa, int dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  R4<real> w;
  const size_t o = (size_t)v.cell_perm[i] * dim;
  w.x = (real)wa[o];
  w.y = (real)wa[o + 1];
  w.z = (dim == 3) ? (real)wa[o + 2] : (real)0;
  w.w = (real)0;
  const_cast<R4<real>*>(v.wmesh)[i] = w;
}

// ------------------------------------------------------------ launchers
template <typename real>
HydroView<real> make_view(amm_ctx* c, double cfl) {
  HydroView<real> v;
  v.dim = c->dim;
  v.mode = c->opt.mesh_motion;
  v.limit = c->opt.limiter;
  v.maxit = c->opt.max_iter;
  v.nboxes = c->nboxes;
  v.n = (int)c->n;
  v.nf = (int)c->nf;
  v.n_ctiles = c->n_ctiles;
  v.n_ftiles = c->n_ftiles;
  v.gamma = c->gamma;
  v.tol = c->opt.riemann_tol;
  v.tol_r = (real)c->opt.riemann_tol;
  v.fixed_acc = (c->opt.precision != AMM_FP64 && !c->opt.fp64_accumulate) ? 1 : 0;
  v.headroom = c->headroom;
  v.update_lanes = (c->update_lanes == 1 || c->update_lanes == 2 || c->update_lanes == 8) ? c->update_lanes : 4;
  v.fmax_bits = c->fmax_bits;
  v.gas = GasC<real>(c->gamma);
  v.cfl = cfl;
  v.dt_box = c->dt_box;
  v.dt_used = c->dt_used;
  v.cour_bits = c->cour_bits;
  v.Q = c->Q;
  v.cw = (R4<real>*)c->cw;
  v.grad = (R4<real>*)c->grad;
  v.pred = (c->opt.mesh_motion == AMM_EULERIAN && c->cwp) ? 1 : 0;
  v.cwp = (R4<real>*)c->cwp;
  v.Apw = (real*)c->Apw;
  v.wmesh = (const R4<real>*)c->wmesh;
  v.cgeo = (const R4<real>*)c->cgeo;
  v.crad = (const real*)c->crad;
  v.cgeo64 = c->cgeo64;

  v.lr = c->lr;
  v.fgeo = (const R4<real>*)c->fgeo;
  v.flux = (R4<real>*)c->flux;
  v.fluxE = (real*)c->fluxE;
  v.csr_off = c->csr_off;
  v.csr = c->csr;
  v.igAB = (const R4<real>*)c->igAB;
  v.ctiles = c->ctiles;
  v.ftiles = c->ftiles;
  v.cell_perm = c->cell_perm;
  v.face_perm = c->face_perm;
  v.partial = c->partial;
  v.totals = c->totals;
  v.box_first_ctile = c->box_first_ctile;
  v.stats = c->stats;
  v.box_status = c->box_status;
  v.regularize = c->opt.regularize;
  v.eta_r = (real)c->opt.eta;
  v.chi_r = (real)c->opt.chi;
  v.wcorr = (R4<real>*)c->wcorr;
  v.entropy = c->opt.entropy;
  v.mach_thresh = c->opt.mach_thresh;
  v.alpha_s = c->opt.alpha_s;
  v.S = c->S;
  v.Aw = (real*)c->Aw;
  v.gradA = (R4<real>*)c->gradA;
  v.fluxS = (real*)c->fluxS;
  v.machf = (real*)c->machf;
  v.ekmax = (real*)c->ekmax;
  v.kept = c->kept;
  v.mlp = c->mlp;
  v.harvest = c->harvest;
  return v;
}

inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

template <typename real>
cudaError_t launch_primitives(amm_ctx* c) {
  auto v = make_view<real>(c, 0.0);
  k_primitives<real><<<nblk(c->n, 256), 256, 0, c->stream>>>(v, nullptr);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_courant(amm_ctx* c) {
  auto v = make_view<real>(c, 0.0);
  cudaError_t e = cudaMemsetAsync(c->cour_bits, 0xff, sizeof(unsigned long long) * c->nboxes, c->stream);
  if (e != cudaSuccess) return e;
  k_courant<real><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gradients(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  // a static mesh's gradient kernel needs the step (k_courant); on a moving
  // mesh it finds the Courant minimum itself
  cudaError_t e = v.pred ? launch_courant<real>(c)
                         : cudaMemsetAsync(c->cour_bits, 0xff, sizeof(unsigned long long) * c->nboxes, c->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(c->fmax_bits, 0, sizeof(unsigned) * FMAX_STRIDE * c->nboxes, c->stream);
  if (e != cudaSuccess) return e;
  if (c->opt.entropy) {
    switch (c->grad_lanes) {
      case 1: k_gradients<real, 1, true><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v); break;
      case 2: k_gradients<real, 2, true><<<c->n_ctiles * 2, CELL_TILE, 0, c->stream>>>(v); break;
      case 8: k_gradients<real, 8, true><<<c->n_ctiles * 8, CELL_TILE, 0, c->stream>>>(v); break;
      default: k_gradients<real, 4, true><<<c->n_ctiles * 4, CELL_TILE, 0, c->stream>>>(v); break;
    }
  } else {
    switch (c->grad_lanes) {
      case 1: k_gradients<real, 1, false><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v); break;
      case 2: k_gradients<real, 2, false><<<c->n_ctiles * 2, CELL_TILE, 0, c->stream>>>(v); break;
      case 8: k_gradients<real, 8, false><<<c->n_ctiles * 8, CELL_TILE, 0, c->stream>>>(v); break;
      default: k_gradients<real, 4, false><<<c->n_ctiles * 4, CELL_TILE, 0, c->stream>>>(v); break;
    }
  }
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_flux(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  const bool b128 = c->flux_block == 128;
  if constexpr (sizeof(real) == 4) {
    // FP32 forms: the persistent chunk kernel (flux_chunks.cu); the learned form adds
    // the deferred proposal kernel
    if (c->opt.precision == AMM_FP32_LEARNED) return launch_flux_learned(c, v);
    return launch_flux_chunks(c, v, false, FluxDefer());
  } else {
    const bool ent = c->opt.entropy != 0;
    if (b128 && ent)
      k_flux<real, 128, true><<<c->n_ftiles * 2, 128, 0, c->stream>>>(v);
    else if (b128)
      k_flux<real, 128, false><<<c->n_ftiles * 2, 128, 0, c->stream>>>(v);
    else if (ent)
      k_flux<real, 256, true><<<c->n_ftiles, 256, 0, c->stream>>>(v);
    else
      k_flux<real, 256, false><<<c->n_ftiles, 256, 0, c->stream>>>(v);
  }
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_update(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  if (c->opt.entropy) {
    switch (c->update_lanes) {
      case 1: k_update<real, 1, true><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v); break;
      case 2: k_update<real, 2, true><<<c->n_ctiles * 2, CELL_TILE, 0, c->stream>>>(v); break;
      case 8: k_update<real, 8, true><<<c->n_ctiles * 8, CELL_TILE, 0, c->stream>>>(v); break;
      default: k_update<real, 4, true><<<c->n_ctiles * 4, CELL_TILE, 0, c->stream>>>(v); break;
    }
  } else {
    switch (c->update_lanes) {
      case 1: k_update<real, 1, false><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v); break;
      case 2: k_update<real, 2, false><<<c->n_ctiles * 2, CELL_TILE, 0, c->stream>>>(v); break;
      case 8: k_update<real, 8, false><<<c->n_ctiles * 8, CELL_TILE, 0, c->stream>>>(v); break;
      default: k_update<real, 4, false><<<c->n_ctiles * 4, CELL_TILE, 0, c->stream>>>(v); break;
    }
  }
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_finish(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  if (cfl < 0.0) {  // totals of the current state, no step
    k_partial_sums<real><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v);
    k_finish<real><<<c->nboxes, FINISH_THREADS, 0, c->stream>>>(v, 0);
  } else {
    k_finish<real><<<c->nboxes, FINISH_THREADS, 0, c->stream>>>(v, 1);
  }
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_set_state(amm_ctx* c, const double* Qa, unsigned long long* bad) {
  auto v = make_view<real>(c, 0.0);
  k_set_state<real><<<nblk(c->n, 256), 256, 0, c->stream>>>(v, Qa, c->dim, bad);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_get_state(amm_ctx* c, double* Qa) {
  auto v = make_view<real>(c, 0.0);
  k_get_state<real><<<nblk(c->n, 256), 256, 0, c->stream>>>(v, Qa, c->dim);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_get_primitives(amm_ctx* c, double* Wa) {
  auto v = make_view<real>(c, 0.0);
  k_get_prims<real><<<nblk(c->n, 256), 256, 0, c->stream>>>(v, Wa, c->dim);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_get_gradients(amm_ctx* c, double* ga) {
  auto v = make_view<real>(c, 0.0);
  k_get_grads<real><<<nblk(c->n, 256), 256, 0, c->stream>>>(v, ga, c->dim);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_get_flux(amm_ctx* c, double* Fa) {
  auto v = make_view<real>(c, 0.0);
  k_get_flux<real><<<nblk(c->nf, 256), 256, 0, c->stream>>>(v, Fa, c->dim);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_set_wmesh(amm_ctx* c, const double* wa) {
  auto v = make_view<real>(c, 0.0);
  k_set_wmesh<real><<<nblk(c->n, 256), 256, 0, c->stream>>>(v, wa, c->dim);
  return cudaGetLastError();
}

#define AMM_INSTANTIATE(real)                                                        \
  template HydroView<real> make_view<real>(amm_ctx*, double);                        \
  template cudaError_t launch_primitives<real>(amm_ctx*);                            \
  template cudaError_t launch_courant<real>(amm_ctx*);                               \
  template cudaError_t launch_gradients<real>(amm_ctx*, double);                     \
  template cudaError_t launch_flux<real>(amm_ctx*, double);                          \
  template cudaError_t launch_update<real>(amm_ctx*, double);                        \
  template cudaError_t launch_finish<real>(amm_ctx*, double);                        \
  template cudaError_t launch_set_state<real>(amm_ctx*, const double*, unsigned long long*); \
  template cudaError_t launch_get_state<real>(amm_ctx*, double*);                    \
  template cudaError_t launch_get_primitives<real>(amm_ctx*, double*);               \
  template cudaError_t launch_get_gradients<real>(amm_ctx*, double*);                \
  template cudaError_t launch_get_flux<real>(amm_ctx*, double*);                     \
  template cudaError_t launch_set_wmesh<real>(amm_ctx*, const double*);

}  // namespace amm
