// Individual power-of-two time steps on a static mesh (Sec. 7.2) with the
// signal-speed criterion of eq. (EqnTiStepIndividual), templated on the bulk
// arithmetic type like hydro.cuh (instantiated in hydro_f64.cu and
// hydro_f32.cu).
//
// A cycle of length dt_max runs in integer ticks of dt_max / 2^D (D =
// max_depth); cell i steps by 2^(D - bin_i) ticks and is active at a tick
// its step divides.  Per tick with active cells the host enqueues:
//
//  k_ind_activate  active cells: W from Q (cw), their walk record, the
//                  active-cell list                          (Sec. 7.2)
//  k_ind_leaf / k_ind_up   per bucket of a uniform-grid pyramid over the
//                  box: the largest sound speed and speed of its cells
//  k_ind_grad      active cells: limited gradients (eq. eqngrad2), the
//                  neighbours entering with their stored W   (Sec. 3.1)
//  k_ind_bins      active cells: dt_i = C min(tau_i, R_i/(c_i+|v_i|)) by a
//                  pruned walk of the pyramid, the new bin (a shorter step
//                  freely, a longer one at most twice the current step and
//                  only where that step starts now), the bin histogram
//                                                             (Sec. 7.1, 7.2)
//  k_ind_faces     faces with an active cell: the active-face list, their
//                  step (the smaller of the two cells') and stamps
//  k_ind_flux      active faces: extrapolation, each side predicted from its
//                  own last activation to the middle of the face's step,
//                  Riemann solve, flux                        (Sec. 3.3)
//  k_ind_update    touched cells: Q -= sum over active faces of
//                  +-dt_f A F (pairwise, conservative; no atomics)
//
// and reads back the bin histogram (64 counters) to find the next tick.
// Lists are built with warp-aggregated atomics; their order is not
// deterministic, but every list item is computed independently and every
// per-cell sum runs in the cell's fixed incidence order, so the results are.
#pragma once

#include "hydro.cuh"

namespace amm {

__device__ __forceinline__ int warp_append(int* counter, bool pred) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (mask == 0u) return -1;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if ((int)lane == leader) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  return pred ? base + __popc(mask & ((1u << lane) - 1u)) : -1;
}

__device__ __forceinline__ long long step_ticks(int depth, int b) { return 1ll << (depth - b); }

// ------------------------------------------------------------- activation
template <typename real>
__global__ void k_ind_activate(HydroView<real> v, IndView d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = i < d.n;
  bool active = false;
  if (in) active = (d.tick & (step_ticks(d.depth, d.bin[i]) - 1)) == 0;
  const int at = warp_append(d.count, active);
  if (!in) return;
  d.act[i] = active ? 1 : 0;
  if (!active) return;
  d.list[at] = i;
  const size_t n = (size_t)v.n;
  const double m = v.Q[i], px = v.Q[n + i], py = v.Q[2 * n + i], pz = v.Q[3 * n + i], E = v.Q[4 * n + i];
  const real P = prims_from_Q(v, i, m, px, py, pz, E);
  if (!(m > 0.0) || !(P > (real)0)) {
    atomicAdd(&v.stats->nonpos, 1ull);
    atomicOr(&v.stats->status, (unsigned)ST_NONPOS);
    atomicOr(v.box_status, (unsigned)ST_NONPOS);
  }
  if (d.signal) {
    // the walk record: position, sound speed, velocity and speed in FP64
    const R4<real> w = v.cw[2 * (size_t)i];
    const double rho = (double)w.x, Pd = (double)P;
    const double vx = (double)w.y, vy = (double)w.z, vz = (double)w.w;
    const double* g = d.gen + 3 * (size_t)i;
    double4 a, b;
    a.x = g[0]; a.y = g[1]; a.z = g[2];
    a.w = sqrt(d.gamma * Pd / rho);
    b.x = vx; b.y = vy; b.z = vz;
    b.w = sqrt(vx * vx + vy * vy + vz * vz);
    const int s = d.cell_slot[i];
    d.rec[2 * (size_t)s] = a;
    d.rec[2 * (size_t)s + 1] = b;
  }
}

// ------------------------------------------------------------ the pyramid
static __global__ void k_ind_leaf(IndView d) {
  const int nb = d.level_off[d.levels - 1];
  const int leaves = (d.dim == 3) ? (1 << (3 * (d.levels - 1))) : (1 << (2 * (d.levels - 1)));
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= leaves) return;
  double cm = 0.0, vm = 0.0;
  for (int s = d.leaf_off[b]; s < d.leaf_off[b + 1]; s++) {
    const double4 a = d.rec[2 * (size_t)s], c = d.rec[2 * (size_t)s + 1];
    cm = fmax(cm, a.w);
    vm = fmax(vm, c.w);
  }
  d.node[nb + b] = make_double2(cm, vm);
}

// all coarser levels by one CTA, finest first
static __global__ void __launch_bounds__(1024) k_ind_up(IndView d) {
  const int ch = (d.dim == 3) ? 8 : 4;
  for (int l = d.levels - 2; l >= 0; l--) {
    const int per = (d.dim == 3) ? (1 << l) * (1 << l) * (1 << l) : (1 << l) * (1 << l);
    const int side = 1 << l;
    for (int b = threadIdx.x; b < per; b += blockDim.x) {
      int ix, iy, iz;
      if (d.dim == 3) {
        ix = b / (side * side); iy = (b / side) % side; iz = b % side;
      } else {
        ix = b / side; iy = b % side; iz = 0;
      }
      const int cs = side * 2;
      double cm = 0.0, vm = 0.0;
      for (int q = 0; q < ch; q++) {
        const int jx = 2 * ix + (q & 1), jy = 2 * iy + ((q >> 1) & 1), jz = 2 * iz + ((q >> 2) & 1);
        const int cb = (d.dim == 3) ? (jx * cs + jy) * cs + jz : jx * cs + jy;
        const double2 c = d.node[d.level_off[l + 1] + cb];
        cm = fmax(cm, c.x);
        vm = fmax(vm, c.y);
      }
      d.node[d.level_off[l] + b] = make_double2(cm, vm);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------- gradients of active cells
template <typename real, int G>
__global__ void __launch_bounds__(CELL_TILE) k_ind_grad(HydroView<real> v, IndView d) {
  constexpr int CELLS = CELL_TILE / G;
  const int count = d.count[0];
  const int lane = (int)threadIdx.x % G;
  for (int blk = blockIdx.x; blk * CELLS < count; blk += gridDim.x) {
    const int idx = blk * CELLS + (int)threadIdx.x / G;
    const bool valid = idx < count;
    const int i = d.list[valid ? idx : 0];
    R4<real> Wi, cg;
    real Pi;
    grad_cell<real, G, false>(v, i, i, valid, lane, Wi, Pi, cg);
  }
}

// ------------------------------------------------------ bins of active cells
// Periodic distance from x to the interval [lo, lo + h] on a circle of length L.
__device__ __forceinline__ double interval_gap(double x, double lo, double h, double L) {
  const double hi = lo + h;
  if (x >= lo && x <= hi) return 0.0;
  const double a = (x < lo) ? lo - x : x - hi;     // direct
  const double b = (x < lo) ? x + L - hi : lo + L - x;  // through the periodic boundary
  return a < b ? a : b;
}

template <typename real>
__global__ void k_ind_bins(HydroView<real> v, IndView d) {
  const int count = d.count[0];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += gridDim.x * blockDim.x) {
    const int i = d.list[idx];
    const R4<real> w = v.cw[2 * (size_t)i];
    const double rho = (double)w.x, P = (double)v.cw[2 * (size_t)i + 1].x;
    const double vx = (double)w.y, vy = (double)w.z, vz = (double)w.w;
    const double ci = sqrt(d.gamma * P / rho);
    const double si = sqrt(vx * vx + vy * vy + vz * vz);
    double cur = (double)v.crad[i] / (ci + si);           // R_i / (c_i + |v_i|)
    if (d.signal) {
      // tau_i = min_j r_ij / (c_i + c_j - v_ij . r_ij / r_ij): a depth-first
      // walk of the pyramid that skips a bucket when even its closest point,
      // its largest sound speed and speed cannot beat the current minimum
      // (r >= gap, signal speed <= c_i + c_max + |v_i| + v_max); the skip test
      // keeps a relative margin of 1e-12, so rounding never drops a pair
      // that would lower the minimum
      const double* gi = d.gen + 3 * (size_t)i;
      const double xi = gi[0], yi = gi[1], zi = gi[2];
      unsigned stack[64];
      int sp = 0;
      stack[sp++] = 0u;                                    // level 0, bucket 0
      const int leaf = d.levels - 1;
      while (sp > 0) {
        const unsigned e = stack[--sp];
        const int l = (int)(e >> 27);
        const int ix = (int)((e >> 18) & 511u), iy = (int)((e >> 9) & 511u), iz = (int)(e & 511u);
        const int side = 1 << l;
        const int b = (d.dim == 3) ? (ix * side + iy) * side + iz : ix * side + iy;
        if (l > 0) {
          const double hx = d.box[0] / side, hy = d.box[1] / side, hz = d.box[2] / side;
          const double gx = interval_gap(xi, ix * hx, hx, d.box[0]);
          const double gy = interval_gap(yi, iy * hy, hy, d.box[1]);
          const double gz = (d.dim == 3) ? interval_gap(zi, iz * hz, hz, d.box[2]) : 0.0;
          const double2 nd = d.node[d.level_off[l] + b];
          const double bound = ci + nd.x + si + nd.y;
          if (!(sqrt(gx * gx + gy * gy + gz * gz) < cur * bound * (1.0 + 1e-12))) continue;
        }
        if (l == leaf) {
          for (int s = d.leaf_off[b]; s < d.leaf_off[b + 1]; s++) {
            if (d.slot_cell[s] == i) continue;
            const double4 a = d.rec[2 * (size_t)s], c = d.rec[2 * (size_t)s + 1];
            double dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
            if (dx > 0.5 * d.box[0]) dx -= d.box[0]; else if (dx < -0.5 * d.box[0]) dx += d.box[0];
            if (dy > 0.5 * d.box[1]) dy -= d.box[1]; else if (dy < -0.5 * d.box[1]) dy += d.box[1];
            if (d.dim == 3) {
              if (dz > 0.5 * d.box[2]) dz -= d.box[2]; else if (dz < -0.5 * d.box[2]) dz += d.box[2];
            } else {
              dz = 0.0;
            }
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double vr = (vx - c.x) * dx + (vy - c.y) * dy + (vz - c.z) * dz;
            const double sig = ci + a.w - vr / r;
            if (sig > 0.0) {
              const double t = r / sig;
              cur = t < cur ? t : cur;
            }
          }
        } else {
          const int nch = (d.dim == 3) ? 8 : 4;
          for (int q = 0; q < nch && sp < 64; q++) {
            const unsigned jx = 2u * ix + (q & 1), jy = 2u * iy + ((q >> 1) & 1), jz = 2u * iz + ((q >> 2) & 1);
            stack[sp++] = ((unsigned)(l + 1) << 27) | (jx << 18) | (jy << 9) | jz;
          }
        }
      }
    }
    const double dti = d.cfl * cur;
    // the largest step dt_max 2^-b not above dt_i
    int b = 0;
    double st = d.dtick * (double)(1ll << d.depth);
    while (st > dti && b <= d.depth) {
      st *= 0.5;
      b++;
    }
    if (b > d.depth) {
      atomicOr(&v.stats->status, (unsigned)ST_DEPTH);
      b = d.depth;
    }
    const int old = d.bin[i];
    int nb = b;
    if (d.tick != 0 && b < old)   // at most twice the step, where that step starts now
      nb = ((d.tick & (step_ticks(d.depth, old - 1) - 1)) == 0) ? old - 1 : old;
    if (nb != old) {
      atomicSub(d.hist + old, 1u);
      atomicAdd(d.hist + nb, 1u);
      d.bin[i] = (signed char)nb;
    }
  }
}

// ------------------------------------------------------------ active faces
template <typename real>
__global__ void k_ind_faces(HydroView<real> v, IndView d) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = k < d.nf;
  int2 e = make_int2(0, 0);
  bool active = false;
  if (in) {
    e = v.lr[k];
    active = d.act[e.x] || d.act[e.y];
  }
  const int at = warp_append(d.count + 1, active);
  if (!active) return;
  d.flist[at] = k;
  d.fstamp[k] = d.stamp;
  d.cstamp[e.x] = d.stamp;   // both writers store the same value
  d.cstamp[e.y] = d.stamp;
  const long long sL = step_ticks(d.depth, d.bin[e.x]), sR = step_ticks(d.depth, d.bin[e.y]);
  d.fdt[k] = (double)(sL < sR ? sL : sR) * d.dtick;
}

// ---------------------------------------------------- fluxes of active faces
template <typename real, int B>
__global__ void __launch_bounds__(B) k_ind_flux(HydroView<real> v, IndView d) {
  const int count = d.count[1];
  for (int blk = blockIdx.x; blk * B < count; blk += gridDim.x) {
    const int idx = blk * B + (int)threadIdx.x;
    const bool valid = idx < count;
    const int k = d.flist[valid ? idx : 0];
    const int2 e = v.lr[k];
    const long long sL = step_ticks(d.depth, d.bin[e.x]), sR = step_ticks(d.depth, d.bin[e.y]);
    const long long sf = sL < sR ? sL : sR;
    const long long t2 = 2 * d.tick + sf;                 // twice the middle of the face's step
    const double hL = (double)(t2 - 2 * (d.tick - (d.tick & (sL - 1)))) * (0.5 * d.dtick);
    const double hR = (double)(t2 - 2 * (d.tick - (d.tick & (sR - 1)))) * (0.5 * d.dtick);
    FaceWork<real> f;
    face_prepare<real, false>(v, k, valid, (real)hL, (real)hR, f);
    face_finish<real, B, false>(v, f, 0, min(B, count - blk * B), false, (real)0);
  }
}

// --------------------------------------------------- the pairwise exchange
template <typename real>
__global__ void k_ind_update(HydroView<real> v, IndView d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n || d.cstamp[i] != d.stamp) return;
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int q = v.csr_off[i]; q < v.csr_off[i + 1]; q++) {
    const int2 e = v.csr[q];
    const int k = e.x >> 1;
    if (d.fstamp[k] != d.stamp) continue;
    const double w = (e.x & 1) ? -d.fdt[k] : d.fdt[k];
    const R4<real> f = v.flux[k];
    s[0] += w * (double)f.x;
    s[1] += w * (double)f.y;
    s[2] += w * (double)f.z;
    s[3] += w * (double)f.w;
    s[4] += w * (double)v.fluxE[k];
  }
  const size_t n = (size_t)d.n;
  for (int a = 0; a < 5; a++) v.Q[a * n + i] -= s[a];
}

// ---------------------------------------------------------------- launchers
template <typename real>
cudaError_t launch_individual_tick(amm_ctx* c, const IndView& d) {
  HydroView<real> v = make_view<real>(c, 0.0);
  v.fixed_acc = 0;                 // per-face steps: the FP64 gather below
  const int grid_c = nblk(c->n, 256);
  k_ind_activate<real><<<grid_c, 256, 0, c->stream>>>(v, d);
  if (d.signal) {
    const int leaves = (d.dim == 3) ? (1 << (3 * (d.levels - 1))) : (1 << (2 * (d.levels - 1)));
    k_ind_leaf<<<nblk(leaves, 256), 256, 0, c->stream>>>(d);
    k_ind_up<<<1, 1024, 0, c->stream>>>(d);
  }
  // list kernels: a fixed grid strides over the list, whose length only the
  // device knows
  const int sms = 152;
  const int g_grad = nblk(c->n, CELL_TILE / 4), g_bins = nblk(c->n, 128), g_flux = nblk(c->nf, 128);
  k_ind_grad<real, 4><<<g_grad < sms * 8 ? g_grad : sms * 8, CELL_TILE, 0, c->stream>>>(v, d);
  k_ind_bins<real><<<g_bins < sms * 8 ? g_bins : sms * 8, 128, 0, c->stream>>>(v, d);
  k_ind_faces<real><<<nblk(c->nf, 256), 256, 0, c->stream>>>(v, d);
  k_ind_flux<real, 128><<<g_flux < sms * 8 ? g_flux : sms * 8, 128, 0, c->stream>>>(v, d);
  k_ind_update<real><<<grid_c, 256, 0, c->stream>>>(v, d);
  return cudaGetLastError();
}

#define AMM_INSTANTIATE_INDIVIDUAL(real) \
  template cudaError_t launch_individual_tick<real>(amm_ctx*, const IndView&);

}  // namespace amm
