// Geometry derived from the face list, once per tessellation (A0), and the
// generator drift (A10).
//
// Per face: unit normal n = (r_R - r_L)/|r_R - r_L| with r_R the periodic
// image, the separation |r_R - r_L|, c = f - (r_L + r_R)/2 and the area.
// Per cell (Sec. 2.3): the volume is the sum of the pyramids over the cell's
// faces with apex at the generator, V_pyr = A (|r_R - r_L|/2) / D; the centre
// of mass is the volume-weighted mean of the pyramid centroids, which lie a
// fraction D/(D+1) of the way from the apex to the face centroid.  The same
// gather yields the closure error |sum_faces A n_out| / sum A (zero for a
// closed cell by the divergence theorem).  All in FP64.
#include "amm_internal.cuh"

namespace amm {

__global__ void k_face_geometry(const Tile* ftiles, const int2* lr, const double* gen, const double* box,
                                const double* area, const double* cen, const int8_t* shift3, R4<double>* fg64) {
  const Tile t = ftiles[blockIdx.x];
  const int k = t.begin + (int)threadIdx.x;
  if (k >= t.end) return;
  const int2 e = lr[k];
  const double* bx = box + 3 * t.box;
  double d[3], m[3];
  for (int a = 0; a < 3; a++) {
    const double rl = gen[3 * (size_t)e.x + a];
    const double rr = gen[3 * (size_t)e.y + a] + (double)shift3[3 * (size_t)k + a] * bx[a];
    d[a] = rr - rl;
    m[a] = 0.5 * (rl + rr);
  }
  const double sep = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  R4<double> g0, g1;
  g0.x = d[0] / sep;
  g0.y = d[1] / sep;
  g0.z = d[2] / sep;
  g0.w = sep;
  g1.x = cen[3 * (size_t)k] - m[0];
  g1.y = cen[3 * (size_t)k + 1] - m[1];
  g1.z = cen[3 * (size_t)k + 2] - m[2];
  g1.w = area[k];
  fg64[2 * (size_t)k] = g0;
  fg64[2 * (size_t)k + 1] = g1;
}

__global__ void k_cell_geometry(int n, int dim, const int* csr_off, const int2* csr, const R4<double>* fg64,
                                R4<double>* cg64, float* closure) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double frac = (double)dim / (double)(dim + 1);
  double V = 0.0, mx = 0.0, my = 0.0, mz = 0.0, cx = 0.0, cy = 0.0, cz = 0.0, asum = 0.0;
  for (int q = csr_off[i]; q < csr_off[i + 1]; q++) {
    const int2 e = csr[q];
    const int k = e.x >> 1;
    const double sg = (e.x & 1) ? -1.0 : 1.0;
    const R4<double> g0 = fg64[2 * (size_t)k], g1 = fg64[2 * (size_t)k + 1];
    const double h = 0.5 * g0.w;
    const double vp = g1.w * h / dim;
    // face centroid relative to the generator of this cell
    const double fx = sg * h * g0.x + g1.x, fy = sg * h * g0.y + g1.y, fz = sg * h * g0.z + g1.z;
    V += vp;
    mx += vp * frac * fx;
    my += vp * frac * fy;
    mz += vp * frac * fz;
    cx += g1.w * sg * g0.x;
    cy += g1.w * sg * g0.y;
    cz += g1.w * sg * g0.z;
    asum += g1.w;
  }
  R4<double> o;
  o.x = V;
  o.y = mx / V;
  o.z = my / V;
  o.w = mz / V;
  cg64[i] = o;
  closure[i] = (float)(sqrt(cx * cx + cy * cy + cz * cz) / (asum > 0.0 ? asum : 1.0));
}

template <typename real>
__global__ void k_cast4(const R4<double>* in, R4<real>* out, size_t count) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const R4<double> a = in[i];
  R4<real> b;
  b.x = (real)a.x;
  b.y = (real)a.y;
  b.z = (real)a.z;
  b.w = (real)a.w;
  out[i] = b;
}

// per-cell constants of the bulk type: 1/V, s - r and the effective radius
// R = (3V/4pi)^(1/3) in 3D, (V/pi)^(1/2) in 2D (eq. EqnTiStep)
template <typename real>
__global__ void k_cell_derived(const R4<double>* cg64, R4<real>* cg, real* crad, R4<real>* cw, int n, int dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R4<double> a = cg64[i];
  R4<real> b;
  b.x = (real)(1.0 / a.x);
  b.y = (real)a.y;
  b.z = (real)a.z;
  b.w = (real)a.w;
  cg[i] = b;
  // s - r in the second half of the cell record (P is written with the state)
  b.x = (real)0;
  cw[2 * (size_t)i + 1] = b;
  crad[i] = (real)((dim == 3) ? cbrt(3.0 * a.x / (4.0 * M_PI)) : sqrt(a.x / M_PI));
}

// Per-incidence record of the gradient (eq. eqngrad2) and of the limiter, in
// the order of the cell->face lists: for incidence q of cell i through face
// k (sign s = +1 if i is the face's left cell, else -1, so s n points out of
// i) and neighbour j, {w = A (c / |d| + s n / 2), 0} and {f - s_i, j}, where
// f - s_i = s |d|/2 n + c - (s_i - r_i) is the limiter's lever arm.  The
// paper's sum over the faces of A ([phi_j - phi_i] c / |d| + (phi_i + phi_j)
// s n / 2) equals the sum of (phi_j - phi_i) w, because a closed cell's
// vector area sum of A s n vanishes: one weight vector per incidence, and a
// uniform field gives exactly zero whatever the rounding.  j is kept as the
// bits of the last real.  Computed once per tessellation from the
// bulk-precision face and cell geometry.
__device__ __forceinline__ float int_bits_real(int j, float) { return __int_as_float(j); }
__device__ __forceinline__ double int_bits_real(int j, double) { return __longlong_as_double((long long)j); }

template <typename real>
__global__ void k_incidence_geometry(int n, const int* csr_off, const int2* csr, const R4<real>* fgeo,
                                     const R4<real>* cgeo, R4<real>* igAB) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R4<real> cg = cgeo[i];
  for (int q = csr_off[i]; q < csr_off[i + 1]; q++) {
    const int2 e = csr[q];
    const int k = e.x >> 1;
    const real sg = (e.x & 1) ? (real)-1 : (real)1;
    const R4<real> G0 = fgeo[2 * (size_t)k];
    const R4<real> G1 = fgeo[2 * (size_t)k + 1];
    const real a_r = G1.w / G0.w;
    const real hs = (real)0.5 * sg * G0.w;
    R4<real> a, b;
    const real a_h = (real)0.5 * G1.w * sg;
    a.x = a_r * G1.x + a_h * G0.x;
    a.y = a_r * G1.y + a_h * G0.y;
    a.z = a_r * G1.z + a_h * G0.z;
    a.w = (real)0;
    b.x = hs * G0.x + G1.x - cg.y;
    b.y = hs * G0.y + G1.y - cg.z;
    b.z = hs * G0.z + G1.z - cg.w;
    b.w = int_bits_real(e.y, (real)0);
    igAB[2 * (size_t)q] = a;
    igAB[2 * (size_t)q + 1] = b;
  }
}

// A10: r_i <- r_i + w_i dt, wrapped into the box; w from the mesh mode, or
// the regularity-corrected velocities of the last step (Sec. 4.1)
__global__ void k_drift(const Tile* ctiles, int mode, int precision, double* gen, const double* box,
                        const double* Q, int n, const void* wmesh, const void* wcorr, double dt) {
  const Tile t = ctiles[blockIdx.x];
  const int i = t.begin + (int)threadIdx.x;
  if (i >= t.end || mode == AMM_EULERIAN) return;
  double w[3];
  if (wcorr) {
    if (precision == AMM_FP64) {
      const R4<double> q = ((const R4<double>*)wcorr)[i];
      w[0] = q.x; w[1] = q.y; w[2] = q.z;
    } else {
      const R4<float> q = ((const R4<float>*)wcorr)[i];
      w[0] = q.x; w[1] = q.y; w[2] = q.z;
    }
  } else if (mode == AMM_LAGRANGIAN) {
    const double m = Q[i];
    for (int a = 0; a < 3; a++) w[a] = Q[(size_t)(a + 1) * n + i] / m;
  } else if (precision == AMM_FP64) {
    const R4<double> q = ((const R4<double>*)wmesh)[i];
    w[0] = q.x; w[1] = q.y; w[2] = q.z;
  } else {
    const R4<float> q = ((const R4<float>*)wmesh)[i];
    w[0] = q.x; w[1] = q.y; w[2] = q.z;
  }
  for (int a = 0; a < 3; a++) {
    const double L = box[3 * t.box + a];
    double x = gen[3 * (size_t)i + a] + w[a] * dt;
    x = fmod(x, L);
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    gen[3 * (size_t)i + a] = x;
  }
}

cudaError_t launch_face_geometry(amm_ctx* c, const double* area, const double* cen, const int8_t* shift3) {
  // fgeo64 temporary in c->fgeo when FP64, else a scratch buffer cast below
  R4<double>* fg64 = nullptr;
  cudaError_t e;
  if (c->is_fp64()) {
    fg64 = (R4<double>*)c->fgeo;
  } else {
    const size_t need = sizeof(R4<double>) * 2 * (size_t)c->nf;
    if (need > c->geo_ws_bytes) {
      if (c->geo_ws) cudaFree(c->geo_ws);
      c->geo_ws = nullptr;
      c->geo_ws_bytes = 0;
      e = cudaMalloc(&c->geo_ws, need);
      if (e != cudaSuccess) return e;
      c->geo_ws_bytes = need;
    }
    fg64 = (R4<double>*)c->geo_ws;
  }
  k_face_geometry<<<c->n_ftiles, FACE_TILE, 0, c->stream>>>(c->ftiles, c->lr, c->gen, c->box, area, cen, shift3,
                                                             fg64);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nb = (int)((c->n + 255) / 256);
  k_cell_geometry<<<nb, 256, 0, c->stream>>>((int)c->n, c->dim, c->csr_off, c->csr, fg64, c->cgeo64, c->closure);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t nfg = 2 * (size_t)c->nf;
  const unsigned nbc = (unsigned)((c->n + 255) / 256);
  if (c->is_fp64()) {
    k_cell_derived<double><<<nbc, 256, 0, c->stream>>>(c->cgeo64, (R4<double>*)c->cgeo, (double*)c->crad,
                                                       (R4<double>*)c->cw, (int)c->n, c->dim);
    k_incidence_geometry<double><<<nbc, 256, 0, c->stream>>>(
        (int)c->n, c->csr_off, c->csr, (const R4<double>*)c->fgeo, (const R4<double>*)c->cgeo, (R4<double>*)c->igAB);
  } else {
    k_cast4<float><<<(unsigned)((nfg + 255) / 256), 256, 0, c->stream>>>(fg64, (R4<float>*)c->fgeo, nfg);
    k_cell_derived<float><<<nbc, 256, 0, c->stream>>>(c->cgeo64, (R4<float>*)c->cgeo, (float*)c->crad,
                                                      (R4<float>*)c->cw, (int)c->n, c->dim);
    k_incidence_geometry<float><<<nbc, 256, 0, c->stream>>>(
        (int)c->n, c->csr_off, c->csr, (const R4<float>*)c->fgeo, (const R4<float>*)c->cgeo, (R4<float>*)c->igAB);
  }
  return cudaGetLastError();
}

cudaError_t launch_drift(amm_ctx* c, double dt) {
  k_drift<<<c->n_ctiles, CELL_TILE, 0, c->stream>>>(c->ctiles, c->opt.mesh_motion, c->opt.precision, c->gen, c->box,
                                                     c->Q, (int)c->n, c->wmesh, c->wcorr, dt);
  return cudaGetLastError();
}

}  // namespace amm
