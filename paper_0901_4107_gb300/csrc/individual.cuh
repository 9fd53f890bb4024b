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
//                  box: the largest c + |v| of its cells and that cell
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
  const long long tick = d.loop->tick;
  bool active = false;
  if (in) active = (tick & (step_ticks(d.depth, d.bin[i]) - 1)) == 0;
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
    d.rec32[2 * (size_t)s] = make_float4((float)a.x, (float)a.y, (float)a.z, (float)a.w);
    d.rec32[2 * (size_t)s + 1] = make_float4((float)b.x, (float)b.y, (float)b.z, (float)b.w);
  }
}

// ------------------------------------------------------------ the pyramid
static __global__ void k_ind_leaf(IndView d) {
  const int nb = d.level_off[d.levels - 1];
  const int leaves = (d.dim == 3) ? (1 << (3 * (d.levels - 1))) : (1 << (2 * (d.levels - 1)));
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= leaves) return;
  // FP32 records, the maximum raised by 1e-5 to cover their rounding (the
  // bounds are used in FP32 only); an empty bucket keeps -1 and a valid slot
  float m = -1.0f;
  int arg = d.leaf_off[b];
  for (int s = d.leaf_off[b]; s < d.leaf_off[b + 1]; s++) {
    const float4 a = d.rec32[2 * (size_t)s], c = d.rec32[2 * (size_t)s + 1];
    if (a.w + c.w > m) {
      m = a.w + c.w;
      arg = s;
    }
  }
  if (arg >= d.n) arg = d.n - 1;
  d.node[nb + b] = make_float2(m >= 0.0f ? m * (1.0f + 1e-5f) : -1.0f, __int_as_float(arg));
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
      float2 m = make_float2(-2.0f, 0.0f);
      for (int q = 0; q < ch; q++) {
        const int jx = 2 * ix + (q & 1), jy = 2 * iy + ((q >> 1) & 1), jz = 2 * iz + ((q >> 2) & 1);
        const int cb = (d.dim == 3) ? (jx * cs + jy) * cs + jz : jx * cs + jy;
        const float2 c = d.node[d.level_off[l + 1] + cb];
        if (c.x > m.x) m = c;
      }
      d.node[d.level_off[l] + b] = m;
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
__device__ __forceinline__ float interval_gap(float x, float lo, float h, float L) {
  const float hi = lo + h;
  if (x >= lo && x <= hi) return 0.0f;
  const float a = (x < lo) ? lo - x : x - hi;       // direct
  const float b = (x < lo) ? x + L - hi : lo + L - x;  // through the periodic boundary
  return a < b ? a : b;
}

// r_ij / (c_i + c_j - v_ij . r_ij / r_ij) for the cell in walk slot s, to the
// nearest periodic image; +inf where the signal speed is not positive
__device__ __forceinline__ double pair_tau(const IndView& d, int s, double xi, double yi, double zi, double ci,
                                          double vx, double vy, double vz) {
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
  return sig > 0.0 ? r / sig : INFINITY;
}

__device__ __forceinline__ double warp_min_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y < x ? y : x;
  }
  return x;
}

// FP32 bounds of a pair's value r / sig, from the FP32 records, with margins
// well above the FP32 rounding of the positions (eps, absolute), of the
// speeds (relative 1e-5) and of the direction of r_ij (|v_ij| eps / r):
// lo <= the FP64 value <= hi; lo = 0 where the pair is too close to bound,
// lo = hi = +inf where the signal speed cannot be positive.
__device__ __forceinline__ void pair_tau_bounds(const IndView& d, int s, float xi, float yi, float zi, float ci,
                                                float vx, float vy, float vz, float eps, float& lo, float& hi) {
  const float4 a = d.rec32[2 * (size_t)s], c = d.rec32[2 * (size_t)s + 1];
  float dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
  const float bx = (float)d.box[0], by = (float)d.box[1], bz = (float)d.box[2];
  if (dx > 0.5f * bx) dx -= bx; else if (dx < -0.5f * bx) dx += bx;
  if (dy > 0.5f * by) dy -= by; else if (dy < -0.5f * by) dy += by;
  if (d.dim == 3) {
    if (dz > 0.5f * bz) dz -= bz; else if (dz < -0.5f * bz) dz += bz;
  } else {
    dz = 0.0f;
  }
  const float r = sqrtf(dx * dx + dy * dy + dz * dz);
  const float rlo = r - 4.0f * eps, rhi = r + 4.0f * eps;
  lo = 0.0f;
  hi = INFINITY;
  if (!(rlo > 0.0f)) return;
  const float ux = vx - c.x, uy = vy - c.y, uz = vz - c.z;
  const float du = sqrtf(ux * ux + uy * uy + uz * uz);
  const float sig = ci + a.w - (ux * dx + uy * dy + uz * dz) / r;
  const float m = 1e-5f * (ci + a.w + du) + 2.0f * du * (4.0f * eps) / rlo;
  const float sig_hi = sig + m, sig_lo = sig - m;
  if (!(sig_hi > 0.0f)) {
    lo = INFINITY;
    return;
  }
  lo = rlo / sig_hi * (1.0f - 1e-5f);
  if (sig_lo > 0.0f) hi = rhi / sig_lo * (1.0f + 1e-5f);
}

// One warp per active cell: dt_i = C min(tau_i, R_i / (c_i + |v_i|)) of
// eq. (EqnTiStepIndividual), then the cell's bin.
//
// tau_i = min_j r_ij / (c_i + c_j - v_ij . r_ij / r_ij) by a walk of the
// pyramid.  A bucket cannot hold a pair below gap / (c_i + |v_i| + max_j
// (c_j + |v_j|)) (r >= gap, signal speed <= c_i + c_j + |v_i - v_j|); the walk
// skips buckets whose bound is not below the current minimum and opens the
// others smallest bound first (the children of a bucket are pushed in order).
// The bounds and a first screen of the pairs run in FP32 with conservative
// margins; every pair that passes the screen is evaluated exactly in FP64, so
// the minimum is the FP64 minimum over all pairs.  It starts from the pairs
// with the fastest cell of every bucket of a coarse level (any pair value
// bounds the minimum).  The lanes split a bucket's children, a leaf's cells
// and the seeds; the stack is per warp in shared memory.
constexpr int BINS_WARPS = 4;

template <typename real>
__global__ void __launch_bounds__(32 * BINS_WARPS) k_ind_bins(HydroView<real> v, IndView d) {
  __shared__ unsigned s_node[BINS_WARPS][64];
  __shared__ float s_lb[BINS_WARPS][64];
  const int lane = (int)threadIdx.x & 31, w = (int)threadIdx.x >> 5;
  const int count = d.count[0];
  const long long tick = d.loop->tick;
  const float eps = 1e-6f * (float)fmax(d.box[0], fmax(d.box[1], d.box[2]));
  for (int idx = blockIdx.x * BINS_WARPS + w; idx < count; idx += gridDim.x * BINS_WARPS) {
    const int i = d.list[idx];
    // the cell's position, sound speed, velocity and speed in FP64: the walk
    // record the activation kernel wrote (one thread per cell), rather than
    // every lane of this warp repeating the FP64 square roots on the narrow
    // FP64 pipe
    double ci, si, vx, vy, vz, xi = 0.0, yi = 0.0, zi = 0.0;
    if (d.signal) {
      const int slot = d.cell_slot[i];
      const double4 ra = d.rec[2 * (size_t)slot], rb = d.rec[2 * (size_t)slot + 1];
      xi = ra.x; yi = ra.y; zi = ra.z; ci = ra.w;
      vx = rb.x; vy = rb.y; vz = rb.z; si = rb.w;
    } else {
      const R4<real> wi = v.cw[2 * (size_t)i];
      const double rho = (double)wi.x, P = (double)v.cw[2 * (size_t)i + 1].x;
      vx = (double)wi.y; vy = (double)wi.z; vz = (double)wi.w;
      ci = sqrt(d.gamma * P / rho);
      si = sqrt(vx * vx + vy * vy + vz * vz);
    }
    double cur = (double)v.crad[i] / (ci + si);           // R_i / (c_i + |v_i|)
    if (d.signal) {
      const float xf = (float)xi, yf = (float)yi, zf = (float)zi;
      const float cf = (float)ci, vxf = (float)vx, vyf = (float)vy, vzf = (float)vz;
      const float minef = (float)(ci + si);
      const float bx = (float)d.box[0], by = (float)d.box[1], bz = (float)d.box[2];
      // the pruning bound curf >= the FP64 minimum: the local term, and upper
      // bounds of the pairs with the fastest cell of each coarse bucket
      float curf = (float)cur * (1.0f + 1e-5f);
      {
        const int ls = d.levels - 1 < 2 ? d.levels - 1 : 2;
        float t = INFINITY;
        for (int b = d.level_off[ls] + lane; b < d.level_off[ls + 1]; b += 32) {
          const int s = __float_as_int(d.node[b].y);
          if (d.slot_cell[s] != i) {
            float lo, hi;
            pair_tau_bounds(d, s, xf, yf, zf, cf, vxf, vyf, vzf, eps, lo, hi);
            t = hi < t ? hi : t;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fminf(t, __shfl_xor_sync(0xffffffffu, t, o));
        curf = t < curf ? t : curf;
      }
      const int leaf = d.levels - 1;
      const int nch = (d.dim == 3) ? 8 : 4;
      // the cell's own leaf bucket and its 3^dim - 1 neighbours first (lane q
      // takes neighbour q), so the walk below starts from a tight bound and
      // skips them
      const int lside = 1 << leaf;
      const int lx = min(lside - 1, max(0, (int)floorf(xf / bx * (float)lside)));
      const int ly = min(lside - 1, max(0, (int)floorf(yf / by * (float)lside)));
      const int lz = (d.dim == 3) ? min(lside - 1, max(0, (int)floorf(zf / bz * (float)lside))) : 0;
      {
        const int nnb = (d.dim == 3) ? 27 : 9;
        int s0 = 0, s1 = 0;
        if (lane < nnb) {
          const int qx = lane % 3 - 1, qy = (lane / 3) % 3 - 1, qz = (d.dim == 3) ? lane / 9 - 1 : 0;
          const int jx = (lx + qx + lside) % lside, jy = (ly + qy + lside) % lside, jz = (lz + qz + lside) % lside;
          const int b = (d.dim == 3) ? (jx * lside + jy) * lside + jz : jx * lside + jy;
          s0 = d.leaf_off[b];
          s1 = d.leaf_off[b + 1];
        }
        float hmin = INFINITY;
        for (int s = s0; s < s1; s++) {
          if (d.slot_cell[s] == i) continue;
          float lo, hi;
          pair_tau_bounds(d, s, xf, yf, zf, cf, vxf, vyf, vzf, eps, lo, hi);
          hmin = hi < hmin ? hi : hmin;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hmin = fminf(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
        curf = hmin < curf ? hmin : curf;
        double t = INFINITY;
        for (int s = s0; s < s1; s++) {
          if (d.slot_cell[s] == i) continue;
          float lo, hi;
          pair_tau_bounds(d, s, xf, yf, zf, cf, vxf, vyf, vzf, eps, lo, hi);
          if (lo < curf) {
            const double ts = pair_tau(d, s, xi, yi, zi, ci, vx, vy, vz);
            t = ts < t ? ts : t;
          }
        }
        t = warp_min_d(t);
        if (t < cur) {
          cur = t;
          const float cu = (float)cur * (1.0f + 1e-5f);
          curf = cu < curf ? cu : curf;
        }
      }
      int sp = 1;
      if (lane == 0) {
        s_node[w][0] = 0u;                                 // level 0, bucket 0
        s_lb[w][0] = 0.0f;
      }
      __syncwarp();
      while (sp > 0) {
        sp--;
        const unsigned e = s_node[w][sp];
        const float lbe = s_lb[w][sp];
        __syncwarp();
        if (!(lbe < curf)) continue;
        const int l = (int)(e >> 27);
        const int ix = (int)((e >> 18) & 511u), iy = (int)((e >> 9) & 511u), iz = (int)(e & 511u);
        const int side = 1 << l;
        if (l == leaf) {
          const int b = (d.dim == 3) ? (ix * side + iy) * side + iz : ix * side + iy;
          // first the FP32 upper bounds tighten curf, then only the pairs
          // whose lower bound stays below it are evaluated in FP64
          const int s0 = d.leaf_off[b], s1 = d.leaf_off[b + 1];
          float hmin = INFINITY;
          for (int s = s0 + lane; s < s1; s += 32) {
            if (d.slot_cell[s] == i) continue;
            float lo, hi;
            pair_tau_bounds(d, s, xf, yf, zf, cf, vxf, vyf, vzf, eps, lo, hi);
            hmin = hi < hmin ? hi : hmin;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) hmin = fminf(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
          curf = hmin < curf ? hmin : curf;
          double t = INFINITY;
          for (int s = s0 + lane; s < s1; s += 32) {
            if (d.slot_cell[s] == i) continue;
            float lo, hi;
            pair_tau_bounds(d, s, xf, yf, zf, cf, vxf, vyf, vzf, eps, lo, hi);
            if (lo < curf) {
              const double ts = pair_tau(d, s, xi, yi, zi, ci, vx, vy, vz);
              t = ts < t ? ts : t;
            }
          }
          t = warp_min_d(t);
          if (t < cur) {
            cur = t;
            const float cu = (float)cur * (1.0f + 1e-5f);
            curf = cu < curf ? cu : curf;
          }
          continue;
        }
        // lane q < nch takes child q: its bound, then its rank among the
        // surviving children (larger bound deeper in the stack)
        const int cside = side * 2;
        bool ok = false;
        float lb = 0.0f;
        unsigned ce = 0u;
        if (lane < nch) {
          const unsigned jx = 2u * ix + (lane & 1), jy = 2u * iy + ((lane >> 1) & 1), jz = 2u * iz + ((lane >> 2) & 1);
          const int cb = (d.dim == 3) ? ((int)jx * cside + (int)jy) * cside + (int)jz : (int)jx * cside + (int)jy;
          const float fast = d.node[d.level_off[l + 1] + cb].x;
          bool near = false;
          if (l + 1 == leaf) {
            // a leaf of the neighbourhood scanned above (periodic distance <= 1)
            const int ax = abs((int)jx - lx), ay = abs((int)jy - ly), az = abs((int)jz - lz);
            near = min(ax, lside - ax) <= 1 && min(ay, lside - ay) <= 1 && min(az, lside - az) <= 1;
          }
          if (fast >= 0.0f && !near) {
            const float hx = bx / (float)cside, hy = by / (float)cside, hz = bz / (float)cside;
            const float gx = interval_gap(xf, (float)jx * hx, hx, bx);
            const float gy = interval_gap(yf, (float)jy * hy, hy, by);
            const float gz = (d.dim == 3) ? interval_gap(zf, (float)jz * hz, hz, bz) : 0.0f;
            const float gap = fmaxf(sqrtf(gx * gx + gy * gy + gz * gz) - eps, 0.0f);
            lb = gap / ((minef + fast) * (1.0f + 1e-5f));
            ok = lb < curf;
            ce = ((unsigned)(l + 1) << 27) | (jx << 18) | (jy << 9) | jz;
          }
        }
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
        int rank = 0;
        for (int q = 0; q < nch; q++) {
          const float lq = __shfl_sync(0xffffffffu, lb, q);
          if (((okm >> q) & 1u) && (lq > lb || (lq == lb && q < lane))) rank++;
        }
        const int nok = __popc(okm);
        if (ok && sp + rank < 64) {
          s_node[w][sp + rank] = ce;
          s_lb[w][sp + rank] = lb;
        }
        __syncwarp();
        sp = sp + nok < 64 ? sp + nok : 64;
      }
    }
    if (lane == 0) {
      const double dti = d.cfl * cur;
      // the largest step dt_max 2^-b not above dt_i, from the exponents and
      // significands (dt_max 2^-b is exact): with dt_max = m1 2^e1 and
      // dt_i = m2 2^e2, b = e1 - e2, plus one if m1 > m2
      const double dtm = d.dtick * (double)(1ll << d.depth);
      int b = 0;
      if (dti < dtm) {
        const long long u1 = __double_as_longlong(dtm), u2 = __double_as_longlong(dti);
        const int e1 = (int)((u1 >> 52) & 0x7ff), e2 = (int)((u2 >> 52) & 0x7ff);
        const long long m1 = u1 & 0xfffffffffffffll, m2 = u2 & 0xfffffffffffffll;
        b = (e2 == 0) ? d.depth + 1 : e1 - e2 + (m1 > m2 ? 1 : 0);   // zero or subnormal: below every bin
      }
      if (b > d.depth) {
        atomicOr(&v.stats->status, (unsigned)ST_DEPTH);
        b = d.depth;
      }
      const int old = d.bin[i];
      int nb = b;
      if (tick != 0 && b < old)   // at most twice the step, where that step starts now
        nb = ((tick & (step_ticks(d.depth, old - 1) - 1)) == 0) ? old - 1 : old;
      if (nb != old) {
        atomicSub(d.hist + old, 1u);
        atomicAdd(d.hist + nb, 1u);
        d.bin[i] = (signed char)nb;
      }
    }
    __syncwarp();
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
  const int stamp = d.loop->stamp;
  d.flist[at] = k;
  d.fstamp[k] = stamp;
  d.cstamp[e.x] = stamp;   // both writers store the same value
  d.cstamp[e.y] = stamp;
  const long long sL = step_ticks(d.depth, d.bin[e.x]), sR = step_ticks(d.depth, d.bin[e.y]);
  d.fdt[k] = (double)(sL < sR ? sL : sR) * d.dtick;
}

// ---------------------------------------------------- fluxes of active faces
template <typename real, int B>
__global__ void __launch_bounds__(B) k_ind_flux(HydroView<real> v, IndView d) {
  const int count = d.count[1];
  const long long tick = d.loop->tick;
  for (int blk = blockIdx.x; blk * B < count; blk += gridDim.x) {
    const int idx = blk * B + (int)threadIdx.x;
    const bool valid = idx < count;
    const int k = d.flist[valid ? idx : 0];
    const int2 e = v.lr[k];
    const long long sL = step_ticks(d.depth, d.bin[e.x]), sR = step_ticks(d.depth, d.bin[e.y]);
    const long long sf = sL < sR ? sL : sR;
    const long long t2 = 2 * tick + sf;                   // twice the middle of the face's step
    const double hL = (double)(t2 - 2 * (tick - (tick & (sL - 1)))) * (0.5 * d.dtick);
    const double hR = (double)(t2 - 2 * (tick - (tick & (sR - 1)))) * (0.5 * d.dtick);
    FaceWork<real> f;
    face_prepare<real, false>(v, k, valid, (real)hL, (real)hR, f);
    face_finish<real, B, false>(v, f, 0, min(B, count - blk * B), false, (real)0);
  }
}

// --------------------------------------------------- the pairwise exchange
template <typename real>
__global__ void k_ind_update(HydroView<real> v, IndView d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const int stamp = d.loop->stamp;
  if (d.cstamp[i] != stamp) return;
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int q = v.csr_off[i]; q < v.csr_off[i + 1]; q++) {
    const int2 e = v.csr[q];
    const int k = e.x >> 1;
    if (d.fstamp[k] != stamp) continue;
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

// ----------------------------------------------------------- the next tick
// One warp: the deepest bin in use (from the histogram), the counters, the
// next tick (the next multiple of the shortest step), a fresh stamp and
// cleared list counters; the cycle's while condition stays set while ticks
// remain, no cell has failed and the sub-step cap is not reached.
static __global__ void k_ind_next(IndView d) {
  const int lane = (int)threadIdx.x;
  const unsigned h0 = lane <= d.depth ? d.hist[lane] : 0u;
  const unsigned h1 = lane + 32 <= d.depth ? d.hist[lane + 32] : 0u;
  const unsigned m0 = __ballot_sync(0xffffffffu, h0 != 0u), m1 = __ballot_sync(0xffffffffu, h1 != 0u);
  if (lane != 0) return;
  const int deepest = m1 ? 32 + 31 - __clz(m1) : (m0 ? 31 - __clz(m0) : 0);
  IndLoop* L = d.loop;
  L->substeps++;
  L->activations += (unsigned long long)d.count[0];
  L->face_fluxes += (unsigned long long)d.count[1];
  L->deepest = deepest > L->deepest ? deepest : L->deepest;
  const long long smin = 1ll << (d.depth - deepest);
  L->tick = (L->tick / smin + 1) * smin;
  L->stamp++;
  d.count[0] = 0;
  d.count[1] = 0;
  const DeviceStats* S = d.stats;
  const bool failed = (S->status & (ST_NEWTON_CAP | ST_NONPOS | ST_DEPTH)) != 0u;
  const bool capped = L->substeps >= L->max_substeps;
  if (capped && L->tick < L->T) atomicOr(&d.stats->status, (unsigned)ST_SUBSTEPS);
  L->go = (L->tick < L->T && !failed && !capped) ? 1 : 0;
  if (d.in_graph) cudaGraphSetConditional(d.handle, (unsigned)L->go);
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
  const int g_grad = nblk(c->n, CELL_TILE / 4), g_bins = nblk(c->n, BINS_WARPS), g_flux = nblk(c->nf, 128);
  k_ind_grad<real, 4><<<g_grad < sms * 8 ? g_grad : sms * 8, CELL_TILE, 0, c->stream>>>(v, d);
  k_ind_bins<real><<<g_bins < sms * 16 ? g_bins : sms * 16, 32 * BINS_WARPS, 0, c->stream>>>(v, d);
  k_ind_faces<real><<<nblk(c->nf, 256), 256, 0, c->stream>>>(v, d);
  k_ind_flux<real, 128><<<g_flux < sms * 8 ? g_flux : sms * 8, 128, 0, c->stream>>>(v, d);
  k_ind_update<real><<<grid_c, 256, 0, c->stream>>>(v, d);
  return cudaGetLastError();
}

#define AMM_INSTANTIATE_INDIVIDUAL(real) \
  template cudaError_t launch_individual_tick<real>(amm_ctx*, const IndView&);

}  // namespace amm
