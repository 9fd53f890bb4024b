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
#include "learned.cuh"
#include "riemann.cuh"

namespace amm {

template <typename real>
__device__ __forceinline__ double box_dt(const HydroView<real>& v, int b) {
  if (v.cfl > 0.0) return v.cfl * __longlong_as_double((long long)v.cour_bits[b]);
  return v.dt_box[b];
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
  v.W[i] = w;
  v.P[i] = P;
  return P;
}

template <typename real>
__global__ void k_primitives(HydroView<real> v, unsigned long long* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const double m = v.Q[i], px = v.Q[v.n + i], py = v.Q[2 * (size_t)v.n + i], pz = v.Q[3 * (size_t)v.n + i];
  const double E = v.Q[4 * (size_t)v.n + i];
  const real P = prims_from_Q(v, i, m, px, py, pz, E);
  if (bad && (!(m > 0.0) || !(P > (real)0))) atomicAdd(bad, 1ull);
}

// ------------------------------------------------------------ A2+A3+A4
template <typename real>
__global__ void __launch_bounds__(CELL_TILE, sizeof(real) == 4 ? 4 : 2) k_gradients(HydroView<real> v) {
  const Tile t = v.ctiles[blockIdx.x];
  const int i = t.begin + (int)threadIdx.x;
  real tc = (real)3.0e38;
  if (i < t.end) {
    const R4<real> Wi = v.W[i];
    const real phi_i[5] = {Wi.x, Wi.y, Wi.z, Wi.w, v.P[i]};
    const R4<real> cg = v.cgeo[i];
    real g[5][3];
    real mx[5], mn[5];
#pragma unroll
    for (int a = 0; a < 5; a++) {
      g[a][0] = g[a][1] = g[a][2] = (real)0;
      mx[a] = mn[a] = phi_i[a];
    }
    const int q0 = v.csr_off[i], q1 = v.csr_off[i + 1];
    for (int q = q0; q < q1; q++) {
      const int2 e = v.csr[q];
      const int k = e.x >> 1;
      const real sg = (e.x & 1) ? (real)-1 : (real)1;
      const R4<real> G0 = v.fgeo[2 * (size_t)k];
      const R4<real> G1 = v.fgeo[2 * (size_t)k + 1];
      const R4<real> Wj = v.W[e.y];
      const real phi_j[5] = {Wj.x, Wj.y, Wj.z, Wj.w, v.P[e.y]};
      // V grad = sum A ([phi_j - phi_i] c / r_ij + (phi_i + phi_j)/2 n_out)
      const real a_r = G1.w / G0.w;
      const real a_h = (real)0.5 * G1.w * sg;
#pragma unroll
      for (int a = 0; a < 5; a++) {
        const real d = (phi_j[a] - phi_i[a]) * a_r;
        const real s = (phi_i[a] + phi_j[a]) * a_h;
        g[a][0] += d * G1.x + s * G0.x;
        g[a][1] += d * G1.y + s * G0.y;
        g[a][2] += d * G1.z + s * G0.z;
        mx[a] = phi_j[a] > mx[a] ? phi_j[a] : mx[a];
        mn[a] = phi_j[a] < mn[a] ? phi_j[a] : mn[a];
      }
    }
    const real invV = cg.x;
#pragma unroll
    for (int a = 0; a < 5; a++) {
      g[a][0] *= invV;
      g[a][1] *= invV;
      g[a][2] *= invV;
    }
    if (v.limit) {
      real alpha[5] = {(real)1, (real)1, (real)1, (real)1, (real)1};
      for (int q = q0; q < q1; q++) {
        const int2 e = v.csr[q];
        const int k = e.x >> 1;
        const real hs = (e.x & 1) ? (real)-0.5 : (real)0.5;
        const R4<real> G0 = v.fgeo[2 * (size_t)k];
        const R4<real> G1 = v.fgeo[2 * (size_t)k + 1];
        // f - s_i = (f - r_i) - (s_i - r_i), f - r_i = |r_ij|/2 n_out + c
        const real fx = hs * G0.w * G0.x + G1.x - cg.y;
        const real fy = hs * G0.w * G0.y + G1.y - cg.z;
        const real fz = hs * G0.w * G0.z + G1.z - cg.w;
#pragma unroll
        for (int a = 0; a < 5; a++) {
          const real dphi = g[a][0] * fx + g[a][1] * fy + g[a][2] * fz;
          real psi = (real)1;
          if (dphi > (real)0)
            psi = (mx[a] - phi_i[a]) / dphi;
          else if (dphi < (real)0)
            psi = (mn[a] - phi_i[a]) / dphi;
          alpha[a] = psi < alpha[a] ? psi : alpha[a];
        }
      }
#pragma unroll
      for (int a = 0; a < 5; a++) {
        g[a][0] *= alpha[a];
        g[a][1] *= alpha[a];
        g[a][2] *= alpha[a];
      }
    }
    R4<real>* go = v.grad + 4 * (size_t)i;
    R4<real> o;
    o.x = g[0][0]; o.y = g[0][1]; o.z = g[0][2]; o.w = g[4][0];
    go[0] = o;
    o.x = g[1][0]; o.y = g[1][1]; o.z = g[1][2]; o.w = g[4][1];
    go[1] = o;
    o.x = g[2][0]; o.y = g[2][1]; o.z = g[2][2]; o.w = g[4][2];
    go[2] = o;
    o.x = g[3][0]; o.y = g[3][1]; o.z = g[3][2]; o.w = (real)0;
    go[3] = o;
    // Courant time R_i / (c_i + |v_i - w_i|)
    real wx = 0, wy = 0, wz = 0;
    if (v.mode == AMM_LAGRANGIAN) {
      wx = Wi.y; wy = Wi.z; wz = Wi.w;
    } else if (v.mode == AMM_EXPLICIT_W) {
      const R4<real> wm = v.wmesh[i];
      wx = wm.x; wy = wm.y; wz = wm.z;
    }
    const real dx = Wi.y - wx, dy = Wi.z - wy, dz = Wi.w - wz;
    const real cs = xsqrt(v.gas.g * phi_i[4] / Wi.x);
    tc = v.crad[i] / (cs + xsqrt(dx * dx + dy * dy + dz * dz));
  }
  // block minimum, then one integer atomic per CTA (positive doubles order
  // like their bit patterns; min is order independent, so this is exact)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const real u = __shfl_xor_sync(0xffffffffu, tc, o);
    tc = u < tc ? u : tc;
  }
  __shared__ real wmin[CELL_TILE / 32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = tc;
  __syncthreads();
  if (threadIdx.x == 0) {
    real m = wmin[0];
    for (int w = 1; w < CELL_TILE / 32; w++) m = wmin[w] < m ? wmin[w] : m;
    const double md = (double)m;
    if (md > 0.0 && md < 1.0e300)
      atomicMin(v.cour_bits + t.box, (unsigned long long)__double_as_longlong(md));
  }
}

// ------------------------------------------------------------ A5+A6+A7
struct FaceStats {
  int iters, guard, vacuum, fail, fallback;
};

template <typename real>
__device__ __forceinline__ void side_state(const HydroView<real>& v, int i, real hsgn, const real* n, real sep,
                                           const real* c, const real* w, real hdt, real* Wp, real* Wpp) {
  const R4<real> Wi = v.W[i];
  const real P = v.P[i];
  const R4<real>* gp = v.grad + 4 * (size_t)i;
  const R4<real> g0 = gp[0], g1 = gp[1], g2 = gp[2], g3 = gp[3];
  const R4<real> cg = v.cgeo[i];
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
  // spatial extrapolation to the face centroid plus half-step prediction with
  // A(W') at the cell centre (gradients are frame independent)
  Wpp[0] = rho + (g0.x * fx + g0.y * fy + g0.z * fz) - hdt * (ux * g0.x + uy * g0.y + uz * g0.z + rho * divv);
  Wpp[1] = ux + (g1.x * fx + g1.y * fy + g1.z * fz) - hdt * (ux * g1.x + uy * g1.y + uz * g1.z + g0.w * ir);
  Wpp[2] = uy + (g2.x * fx + g2.y * fy + g2.z * fz) - hdt * (ux * g2.x + uy * g2.y + uz * g2.z + g1.w * ir);
  Wpp[3] = uz + (g3.x * fx + g3.y * fy + g3.z * fz) - hdt * (ux * g3.x + uy * g3.y + uz * g3.z + g2.w * ir);
  Wpp[4] = P + (g0.w * fx + g1.w * fy + g2.w * fz) -
           hdt * ((real)v.gamma * P * divv + ux * g0.w + uy * g1.w + uz * g2.w);
}

template <typename real, bool LEARNED>
__global__ void __launch_bounds__(FACE_TILE) k_flux(HydroView<real> v) {
  const Tile t = v.ftiles[blockIdx.x];
  const int k0 = t.begin + (int)threadIdx.x;
  const bool valid = k0 < t.end;
  const int k = valid ? k0 : t.begin;
  const GasC<real>& G = v.gas;
  const real hdt = (real)(0.5 * box_dt(v, t.box));
  const int2 lr = v.lr[k];
  const R4<real> G0 = v.fgeo[2 * (size_t)k];
  const R4<real> G1 = v.fgeo[2 * (size_t)k + 1];
  const real n[3] = {G0.x, G0.y, G0.z};
  const real sep = G0.w;
  const real c[3] = {G1.x, G1.y, G1.z};
  const real A = G1.w;
  // face velocity: mean of the generators' velocities plus the normal motion
  // of the face centroid from their relative motion about the midpoint
  real w[3] = {(real)0, (real)0, (real)0};
  if (v.mode != AMM_EULERIAN) {
    real wl[3], wr[3];
    if (v.mode == AMM_LAGRANGIAN) {
      const R4<real> a = v.W[lr.x], b = v.W[lr.y];
      wl[0] = a.y; wl[1] = a.z; wl[2] = a.w;
      wr[0] = b.y; wr[1] = b.z; wr[2] = b.w;
    } else {
      const R4<real> a = v.wmesh[lr.x], b = v.wmesh[lr.y];
      wl[0] = a.x; wl[1] = a.y; wl[2] = a.z;
      wr[0] = b.x; wr[1] = b.y; wr[2] = b.z;
    }
    const real rot = ((wl[0] - wr[0]) * c[0] + (wl[1] - wr[1]) * c[1] + (wl[2] - wr[2]) * c[2]) / sep;
#pragma unroll
    for (int d = 0; d < 3; d++) w[d] = (real)0.5 * (wl[d] + wr[d]) + rot * n[d];
  }
  real WpL[5], WppL[5], WpR[5], WppR[5];
  side_state(v, lr.x, (real)0.5, n, sep, c, w, hdt, WpL, WppL);
  side_state(v, lr.y, (real)-0.5, n, sep, c, w, hdt, WpR, WppR);
  FaceStats st = {0, 0, 0, 0, 0};
  if (!(WppL[0] > (real)0) || !(WppL[4] > (real)0) || !(WppR[0] > (real)0) || !(WppR[4] > (real)0)) {
#pragma unroll
    for (int a = 0; a < 5; a++) {
      WppL[a] = WpL[a];
      WppR[a] = WpR[a];
    }
    st.fallback = 1;
  }
  // rotate: normal component and transverse vector
  const real uL = WppL[1] * n[0] + WppL[2] * n[1] + WppL[3] * n[2];
  const real uR = WppR[1] * n[0] + WppR[2] * n[1] + WppR[3] * n[2];
  real guess = (real)0;
  bool have_guess = false;
  if constexpr (LEARNED) {
    guess = learned_guess<real>(v.mlp, WppL[0], WppL[4], uL, WppR[0], WppR[4], uR, G);
    have_guess = true;
  }
  real rhoF, uF, pF;
  RiemannInfo info;
  const int side = riemann_sample(WppL[0], uL, WppL[4], WppR[0], uR, WppR[4], G, v.tol, v.maxit, have_guess,
                                  guess, rhoF, uF, pF, info);
  st.iters = info.iters;
  st.guard = info.guard;
  st.vacuum = info.vacuum;
  st.fail = info.fail;
  const real* Wt = side ? WppR : WppL;
  const real ut = side ? uR : uL;
  real vlab[3];
#pragma unroll
  for (int d = 0; d < 3; d++) vlab[d] = uF * n[d] + (Wt[1 + d] - ut * n[d]) + w[d];
  const real v2 = vlab[0] * vlab[0] + vlab[1] * vlab[1] + vlab[2] * vlab[2];
  const real vn = vlab[0] * n[0] + vlab[1] * n[1] + vlab[2] * n[2];
  const real mflux = rhoF * uF;
  if (valid) {
    R4<real> f;
    f.x = A * mflux;
    f.y = A * (mflux * vlab[0] + pF * n[0]);
    f.z = A * (mflux * vlab[1] + pF * n[1]);
    f.w = A * (mflux * vlab[2] + pF * n[2]);
    v.flux[k] = f;
    v.fluxE[k] = A * (((real)0.5 * rhoF * v2 + pF * G.inv_gm1) * uF + pF * vn);
  }
  // statistics: block histogram in shared memory, then a few global atomics
  __shared__ unsigned int sh[16 + 6];
  if (threadIdx.x < 22) sh[threadIdx.x] = 0;
  __syncthreads();
  if (valid) {
    atomicAdd(&sh[st.iters < 15 ? st.iters : 15], 1u);
    atomicAdd(&sh[16], (unsigned)st.iters);
    if (st.guard) atomicAdd(&sh[17], 1u);
    if (st.vacuum) atomicAdd(&sh[18], 1u);
    if (st.fail) atomicAdd(&sh[19], 1u);
    if (st.fallback) atomicAdd(&sh[20], 1u);
    atomicMax(&sh[21], (unsigned)st.iters);
  }
  __syncthreads();
  DeviceStats* S = v.stats;
  if (threadIdx.x < 16) {
    if (sh[threadIdx.x]) atomicAdd(&S->hist[threadIdx.x], (unsigned long long)sh[threadIdx.x]);
  } else if (threadIdx.x == 16) {
    atomicAdd(&S->newton_iters, (unsigned long long)sh[16]);
    atomicAdd(&S->faces, (unsigned long long)(t.end - t.begin));
  } else if (threadIdx.x == 17) {
    if (sh[17]) atomicAdd(&S->guard, (unsigned long long)sh[17]);
  } else if (threadIdx.x == 18) {
    if (sh[18]) atomicAdd(&S->vacuum, (unsigned long long)sh[18]);
  } else if (threadIdx.x == 19) {
    if (sh[19]) {
      atomicAdd(&S->newton_fail, (unsigned long long)sh[19]);
      atomicOr(&S->status, (unsigned)ST_NEWTON_CAP);
    }
  } else if (threadIdx.x == 20) {
    if (sh[20]) atomicAdd(&S->fallback, (unsigned long long)sh[20]);
  } else if (threadIdx.x == 21) {
    atomicMax(&S->newton_max, sh[21]);
  }
}

// ------------------------------------------------------------ A8+A1+A9
template <typename real>
__global__ void __launch_bounds__(CELL_TILE) k_update(HydroView<real> v) {
  const Tile t = v.ctiles[blockIdx.x];
  const int i = t.begin + (int)threadIdx.x;
  double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  unsigned nonpos = 0;
  if (i < t.end) {
    const double dt = box_dt(v, t.box);
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int q0 = v.csr_off[i], q1 = v.csr_off[i + 1];
    for (int e = q0; e < q1; e++) {
      const int2 r = v.csr[e];
      const int k = r.x >> 1;
      const R4<real> f = v.flux[k];
      const double fe = (double)v.fluxE[k];
      if (r.x & 1) {
        acc[0] -= (double)f.x; acc[1] -= (double)f.y; acc[2] -= (double)f.z; acc[3] -= (double)f.w;
        acc[4] -= fe;
      } else {
        acc[0] += (double)f.x; acc[1] += (double)f.y; acc[2] += (double)f.z; acc[3] += (double)f.w;
        acc[4] += fe;
      }
    }
    const size_t n = (size_t)v.n;
#pragma unroll
    for (int a = 0; a < 5; a++) {
      q[a] = v.Q[a * n + i] - dt * acc[a];
      v.Q[a * n + i] = q[a];
    }
    const real P = prims_from_Q(v, i, q[0], q[1], q[2], q[3], q[4]);
    nonpos = (!(q[0] > 0.0) || !(P > (real)0)) ? 1u : 0u;
  }
  // per-tile FP64 sums in a fixed tree order (bit reproducible)
  __shared__ double red[5][CELL_TILE];
#pragma unroll
  for (int a = 0; a < 5; a++) red[a][threadIdx.x] = q[a];
  __syncthreads();
  for (int s = CELL_TILE / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int a = 0; a < 5; a++) red[a][threadIdx.x] += red[a][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) v.partial[5 * (size_t)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
  const unsigned bad = __syncthreads_count(nonpos);
  if (threadIdx.x == 0 && bad) {
    atomicAdd(&v.stats->nonpos, (unsigned long long)bad);
    atomicOr(&v.stats->status, (unsigned)ST_NONPOS);
  }
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
  if (threadIdx.x < 5) v.partial[5 * (size_t)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// one CTA per box: ordered sum of the box's tile partials; time step record
template <typename real>
__global__ void k_finish(HydroView<real> v, int count_step) {
  const int b = blockIdx.x;
  const int t0 = v.box_first_ctile[b], t1 = v.box_first_ctile[b + 1];
  __shared__ double red[5][128];
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int tt = t0 + (int)threadIdx.x; tt < t1; tt += 128)
#pragma unroll
    for (int a = 0; a < 5; a++) s[a] += v.partial[5 * (size_t)tt + a];
#pragma unroll
  for (int a = 0; a < 5; a++) red[a][threadIdx.x] = s[a];
  __syncthreads();
  for (int st = 64; st > 0; st >>= 1) {
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
}

// ------------------------------------------------------------ layout moves
template <typename real>
__global__ void k_set_state(HydroView<real> v, const double* Qa, int dim, unsigned long long* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int nv = dim + 2;
  const double* q = Qa + (size_t)i * nv;
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
  if (!(m > 0.0) || !(P > (real)0)) atomicAdd(bad, 1ull);
}

template <typename real>
__global__ void k_get_state(HydroView<real> v, double* Qa, int dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int nv = dim + 2;
  const size_t n = (size_t)v.n;
  double* q = Qa + (size_t)i * nv;
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
  const R4<real> w = v.W[i];
  double* o = Wa + (size_t)i * nv;
  o[0] = w.x;
  o[1] = w.y;
  o[2] = w.z;
  if (dim == 3) o[3] = w.w;
  o[dim + 1] = v.P[i];
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
  double* o = ga + (size_t)i * (dim + 2) * dim;
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
  double* o = Fa + (size_t)k * (dim + 2);
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
  w.x = (real)wa[(size_t)i * dim];
  w.y = (real)wa[(size_t)i * dim + 1];
  w.z = (dim == 3) ? (real)wa[(size_t)i * dim + 2] : (real)0;
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
  v.gamma = c->gamma;
  v.tol = c->opt.riemann_tol;
  v.gas = GasC<real>(c->gamma);
  v.cfl = cfl;
  v.dt_box = c->dt_box;
  v.dt_used = c->dt_used;
  v.cour_bits = c->cour_bits;
  v.Q = c->Q;
  v.W = (R4<real>*)c->W;
  v.P = (real*)c->P;
  v.grad = (R4<real>*)c->grad;
  v.wmesh = (const R4<real>*)c->wmesh;
  v.cgeo = (const R4<real>*)c->cgeo;
  v.cgeo64 = c->cgeo64;
  v.crad = (const real*)c->crad;
  v.lr = c->lr;
  v.fgeo = (const R4<real>*)c->fgeo;
  v.flux = (R4<real>*)c->flux;
  v.fluxE = (real*)c->fluxE;
  v.csr_off = c->csr_off;
  v.csr = c->csr;
  v.ctiles = c->ctiles;
  v.ftiles = c->ftiles;
  v.partial = c->partial;
  v.totals = c->totals;
  v.box_first_ctile = c->box_first_ctile;
  v.stats = c->stats;
  v.mlp = c->mlp;
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
cudaError_t launch_gradients(amm_ctx* c) {
  auto v = make_view<real>(c, 0.0);
  cudaError_t e = cudaMemsetAsync(c->cour_bits, 0xff, sizeof(unsigned long long) * c->nboxes, c->stream);
  if (e != cudaSuccess) return e;
  k_gradients<real><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_flux(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  if (c->opt.precision == AMM_FP32_LEARNED) {
    if constexpr (sizeof(real) == 4) {
      k_flux<real, true><<<c->n_ftiles, FACE_TILE, 0, c->stream>>>(v);
    } else {
      return cudaErrorInvalidValue;
    }
  } else {
    k_flux<real, false><<<c->n_ftiles, FACE_TILE, 0, c->stream>>>(v);
  }
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_update(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  k_update<real><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_finish(amm_ctx* c, double cfl) {
  auto v = make_view<real>(c, cfl);
  if (cfl < 0.0) {  // totals of the current state, no step
    k_partial_sums<real><<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(v);
    k_finish<real><<<c->nboxes, 128, 0, c->stream>>>(v, 0);
  } else {
    k_finish<real><<<c->nboxes, 128, 0, c->stream>>>(v, 1);
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
  template cudaError_t launch_gradients<real>(amm_ctx*);                             \
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
