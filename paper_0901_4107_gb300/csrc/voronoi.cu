// Voronoi tessellation of a periodic box on the GPU (Sec. 2): the face list
// (two cells, periodic image of the right cell, area, centroid) that the hydro
// update consumes, built from the generators alone.
//
// Each cell is the intersection of the half-spaces bounded by the bisectors
// between its generator and nearby generators (and their periodic images),
// the definition of a Voronoi cell.  Candidates come from a uniform grid of
// bins in shells of growing Chebyshev radius; the search ends once the shell
// boundary is farther from the generator than twice the largest distance to a
// vertex of the current cell -- no generator beyond can cut it (the
// completeness radius of Sec. 2.4).
//
// 3D: one warp per cell.  The convex cell is held in shared memory as its
// planes and its dual triangulation: each vertex is a triangle (a, b, c) of
// three planes, oriented so that triangles sharing two planes list them in
// opposite order.  Cutting by a plane marks the vertices outside it (lanes
// over vertices), turns every edge between a marked and a kept vertex into a
// new vertex on the plane (lanes over the marked vertices), and drops the
// marked ones; vertex positions are the intersections of their three planes.
// A face is the cycle of vertices around its plane; its area and centroid are
// summed over a fan.  2D: one lane per cell keeps the cell polygon as its
// cyclic list of lines.
//
// Faces of (numerically) zero area are dropped, as are planes that only touch
// the cell.  Generators must lie in [0, box).  Results do not depend on the
// launch shape: every cell is built by the same sequence of cuts (candidates
// in bin order, bins in a fixed order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "amm.h"

namespace amm {
namespace vor {

constexpr int WARPS = 2;      // cells per CTA (3D)
constexpr int MAXP = 128;     // planes per cell: 6 of the box + the cutting bisectors
constexpr int MAXT = 384;     // vertex slots (dual triangles), dead ones included
constexpr int MAXC = 192;     // candidates gathered per pass
constexpr int MAXFV = 48;     // vertices of one face
constexpr int MAXHF = 64;     // output half-faces per cell (3D); 2D uses 32

// error codes, as the host tessellator's
constexpr int E_CAPACITY = -1, E_VANISHED = -2, E_INCOMPLETE = -3, E_OPEN = -4, E_FACES = -6, E_CANDIDATES = -7;

struct Grid {
  int dim, n;
  int nb[3];
  double bs[3], box[3];
  const double* pts;         // [n][dim]
  const int* bin_start;      // [nbins + 1]
  const int* bin_pts;        // [n] point indices by bin, ascending within a bin
};

struct HalfFace {
  int j;                     // neighbour generator
  signed char s[4];          // periodic image of the neighbour (box lengths), s[3] unused
  double area;               // area (length in 2D)
  double cen[3];             // centroid relative to this cell's generator
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ int bin_coord(double x, double bs, int nb) {
  int q = (int)floor(x / bs);
  return q < 0 ? 0 : (q >= nb ? nb - 1 : q);
}

// ------------------------------------------------------------ the bin grid
__global__ void k_bin_count(Grid G, int* binof, int* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
  int b[3] = {0, 0, 0};
  for (int d = 0; d < G.dim; d++) b[d] = bin_coord(G.pts[(size_t)i * G.dim + d], G.bs[d], G.nb[d]);
  const int bin = (b[2] * G.nb[1] + b[1]) * G.nb[0] + b[0];
  binof[i] = bin;
  atomicAdd(count + bin, 1);
}

// exclusive scan of count[0..m) into start[0..m], one CTA of 1024 threads
__global__ void k_scan(const int* count, int* start, int m) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (m + 1023) / 1024;
  const int lo = t * per, hi = lo + per < m ? lo + per : m;
  int s = 0;
  for (int k = lo; k < hi; k++) s += count[k];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = t ? part[t - 1] : 0;
  for (int k = lo; k < hi; k++) {
    start[k] = run;
    run += count[k];
  }
  if (t == 1023) start[m] = part[1023];
}

__global__ void k_bin_fill(Grid G, const int* binof, int* cursor, int* bin_pts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
  bin_pts[atomicAdd(cursor + binof[i], 1)] = i;
}

// ascending point index within each bin (bins hold a few points)
__global__ void k_bin_sort(const int* bin_start, int* bin_pts, int m) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m) return;
  const int lo = bin_start[b], hi = bin_start[b + 1];
  for (int k = lo + 1; k < hi; k++) {
    const int v = bin_pts[k];
    int q = k - 1;
    while (q >= lo && bin_pts[q] > v) {
      bin_pts[q + 1] = bin_pts[q];
      q--;
    }
    bin_pts[q + 1] = v;
  }
}

// ------------------------------------------------------------- 3D, a warp per cell
struct Cell3 {
  double pn[MAXP][4];          // the plane n.x = h (x relative to the generator): for a bisector n is the
                               // vector to the neighbour's image and h = |n|^2 / 2; for the box, unit n
  float pnf[MAXP][4];          // the same in FP32
  int pj[MAXP];                // neighbour (-1: a face of the initial box)
  signed char ps[MAXP][4];     // its periodic image
  unsigned char tri[MAXT][4];  // a vertex: planes a, b, c; [3] = 1 while it exists
  float tvf[MAXT][4];          // its position in FP32 and |v| (the FP64 position is recomputed from the
                               // three planes where it is needed: close side tests, the final faces)
  double cx[MAXC][3];          // candidates: image position relative to the generator
  double cd2[MAXC];
  float cd2f[MAXC];
  int cj[MAXC];
  signed char cs[MAXC][4];
  short ord[MAXC];             // candidates by distance
  int mk[MAXT];                // the vertices a cut removes
  int np, nt, nc, nm;
};

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// the point on planes a, b, c
__device__ __forceinline__ void vertex3(const Cell3& C, int a, int b, int c, double* v) {
  const double* na = C.pn[a];
  const double* nb = C.pn[b];
  const double* nc = C.pn[c];
  double bc[3], ca[3], ab[3];
  cross3(nb, nc, bc);
  cross3(nc, na, ca);
  cross3(na, nb, ab);
  const double inv = 1.0 / dot3(na, bc);
  for (int d = 0; d < 3; d++) v[d] = (na[3] * bc[d] + nb[3] * ca[d] + nc[3] * ab[d]) * inv;
}

// The point on planes a, b, c in FP32, when the three are well conditioned
// (|det| >= 0.1 |n_a||n_b||n_c|, so the FP32 position is good to a few 1e-7
// of |v|, far inside the side tests' margin); false otherwise.
__device__ __forceinline__ bool vertex3f(const Cell3& C, int a, int b, int c, float* v) {
  const float* na = C.pnf[a];
  const float* nb = C.pnf[b];
  const float* nc = C.pnf[c];
  const float bc[3] = {nb[1] * nc[2] - nb[2] * nc[1], nb[2] * nc[0] - nb[0] * nc[2], nb[0] * nc[1] - nb[1] * nc[0]};
  const float ca[3] = {nc[1] * na[2] - nc[2] * na[1], nc[2] * na[0] - nc[0] * na[2], nc[0] * na[1] - nc[1] * na[0]};
  const float ab[3] = {na[1] * nb[2] - na[2] * nb[1], na[2] * nb[0] - na[0] * nb[2], na[0] * nb[1] - na[1] * nb[0]};
  const float det = na[0] * bc[0] + na[1] * bc[1] + na[2] * bc[2];
  const float la = na[0] * na[0] + na[1] * na[1] + na[2] * na[2];
  const float lb = nb[0] * nb[0] + nb[1] * nb[1] + nb[2] * nb[2];
  const float lc = nc[0] * nc[0] + nc[1] * nc[1] + nc[2] * nc[2];
  if (!(det * det >= 0.01f * la * lb * lc)) return false;
  const float inv = 1.0f / det;
  for (int d = 0; d < 3; d++) v[d] = (na[3] * bc[d] + nb[3] * ca[d] + nc[3] * ab[d]) * inv;
  return true;
}

// the FP32 copy of vertex t from its FP64 position v: position and |v|
__device__ __forceinline__ void set_f32(Cell3& C, int t, const double* v) {
  C.tvf[t][0] = (float)v[0];
  C.tvf[t][1] = (float)v[1];
  C.tvf[t][2] = (float)v[2];
  C.tvf[t][3] = sqrtf(C.tvf[t][0] * C.tvf[t][0] + C.tvf[t][1] * C.tvf[t][1] + C.tvf[t][2] * C.tvf[t][2]);
}

__device__ __forceinline__ bool has_edge(const unsigned char* t, int u, int w) {
  return (t[0] == u && t[1] == w) || (t[1] == u && t[2] == w) || (t[2] == u && t[0] == w);
}

// drop dead vertex slots (dest <= source, a round reads before it writes)
__device__ void compact3(Cell3& C, int lane) {
  int w = 0;
  for (int base = 0; base < C.nt; base += 32) {
    const int t = base + lane;
    const bool live = t < C.nt && C.tri[t][3];
    unsigned char tr[4] = {0, 0, 0, 0};
    float vf[4] = {0, 0, 0, 0};
    if (live) {
      for (int k = 0; k < 4; k++) tr[k] = C.tri[t][k];
      for (int d = 0; d < 4; d++) vf[d] = C.tvf[t][d];
    }
    const unsigned m = __ballot_sync(0xffffffffu, live);
    __syncwarp();
    if (live) {
      const int dst = w + __popc(m & ((1u << lane) - 1u));
      for (int k = 0; k < 4; k++) C.tri[dst][k] = tr[k];
      for (int d = 0; d < 4; d++) C.tvf[dst][d] = vf[d];
    }
    w += __popc(m);
    __syncwarp();
  }
  if (lane == 0) C.nt = w;
  __syncwarp();
}

// Is vertex t outside {x : n.x <= h} by more than eps (eps scaled with |n|)?
// An FP32 screen decides the clear cases (its error, a few 1e-7 of
// |n||v| + |h|, is far below its margin); the rest in FP64.
__device__ __forceinline__ bool outside(const Cell3& C, int t, const double* n, double h, const float* nf,
                                        double eps) {
  const float* v = C.tvf[t];
  const float d = nf[0] * v[0] + nf[1] * v[1] + nf[2] * v[2] - nf[3];
  const float tol = 1e-5f * (sqrtf(nf[0] * nf[0] + nf[1] * nf[1] + nf[2] * nf[2]) * v[3] + fabsf(nf[3]));
  if (d > tol) return true;
  if (d < -tol) return false;
  double x[3];
  vertex3(C, C.tri[t][0], C.tri[t][1], C.tri[t][2], x);
  return dot3(x, n) - h > eps;
}

// Cut the cell by {x : n.x <= h}.  Returns 0 if the plane misses the cell
// (within eps), 1 after a cut, a negative code on overflow or if the cell
// vanished.  R2 (the largest squared vertex distance) is updated.
__device__ int cut3(Cell3& C, int lane, const double* n, double h, int j, const signed char* s, double eps,
                    float& R2) {
  const float nf[4] = {(float)n[0], (float)n[1], (float)n[2], (float)h};
  // vertices outside the plane
  int nm = 0;
  for (int base = 0; base < C.nt; base += 32) {
    const int t = base + lane;
    bool out = false;
    if (t < C.nt && C.tri[t][3]) out = outside(C, t, n, h, nf, eps);
    const unsigned m = __ballot_sync(0xffffffffu, out);
    if (out) C.mk[nm + __popc(m & ((1u << lane) - 1u))] = t;
    nm += __popc(m);
  }
  __syncwarp();
  if (nm == 0) return 0;
  if (C.np >= MAXP) return E_CAPACITY;
  if (C.nt + 3 * nm > MAXT) {
    compact3(C, lane);
    // the marked indices moved: mark again
    nm = 0;
    for (int base = 0; base < C.nt; base += 32) {
      const int t = base + lane;
      bool out = false;
      if (t < C.nt) out = outside(C, t, n, h, nf, eps);
      const unsigned m = __ballot_sync(0xffffffffu, out);
      if (out) C.mk[nm + __popc(m & ((1u << lane) - 1u))] = t;
      nm += __popc(m);
    }
    __syncwarp();
    if (C.nt + 3 * nm > MAXT) return E_CAPACITY;
  }
  const int q = C.np;
  if (lane == 0) {
    for (int d = 0; d < 3; d++) C.pn[q][d] = n[d];
    C.pn[q][3] = h;
    for (int d = 0; d < 4; d++) C.pnf[q][d] = nf[d];
    C.pj[q] = j;
    for (int d = 0; d < 4; d++) C.ps[q][d] = s[d];
    C.np = q + 1;
  }
  __syncwarp();
  // every edge from a removed vertex to a kept one becomes a vertex on the
  // new plane: (u, w, q) for the removed vertex's edge (u, w)
  int nt = C.nt;
  for (int base = 0; base < nm; base += 32) {
    const int m = base + lane;
    unsigned char e[3][2];
    bool bnd[3] = {false, false, false};
    int cnt = 0;
    if (m < nm) {
      const unsigned char* t = C.tri[C.mk[m]];
      e[0][0] = t[0]; e[0][1] = t[1];
      e[1][0] = t[1]; e[1][1] = t[2];
      e[2][0] = t[2]; e[2][1] = t[0];
      for (int k = 0; k < 3; k++) {
        bool inner = false;
        for (int m2 = 0; m2 < nm && !inner; m2++) inner = has_edge(C.tri[C.mk[m2]], e[k][1], e[k][0]);
        bnd[k] = !inner;
        cnt += bnd[k] ? 1 : 0;
      }
    }
    int pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += y;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    int slot = nt + pre - cnt;
    if (m < nm) {
      for (int k = 0; k < 3; k++) {
        if (!bnd[k]) continue;
        C.tri[slot][0] = e[k][0];
        C.tri[slot][1] = e[k][1];
        C.tri[slot][2] = (unsigned char)q;
        float vf[3];
        if (vertex3f(C, e[k][0], e[k][1], q, vf)) {
          C.tri[slot][3] = 1;
          for (int d = 0; d < 3; d++) C.tvf[slot][d] = vf[d];
          C.tvf[slot][3] = sqrtf(vf[0] * vf[0] + vf[1] * vf[1] + vf[2] * vf[2]);
        } else {
          double v[3];
          vertex3(C, e[k][0], e[k][1], q, v);
          C.tri[slot][3] = 1;
          set_f32(C, slot, v);
        }
        slot++;
      }
    }
    nt += total;
  }
  __syncwarp();
  for (int m = lane; m < nm; m += 32) C.tri[C.mk[m]][3] = 0;
  if (lane == 0) C.nt = nt;
  __syncwarp();
  float r = 0.0f;
  int live = 0;
  for (int t = lane; t < nt; t += 32)
    if (C.tri[t][3]) {
      r = fmaxf(r, C.tvf[t][3]);
      live++;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    live += __shfl_xor_sync(0xffffffffu, live, o);
  }
  R2 = r * r * (1.0f + 1e-5f);           // an upper bound of the largest squared vertex distance
  return live >= 4 ? 1 : E_VANISHED;
}

// Gathers the points of bins [q0, q1) of the shell (bins of the (2s+1)^dim
// cube around bin b at Chebyshev distance >= s0, in cube order) into the
// candidate buffer, from position `at`; lanes take bins.  Returns the new
// count, or -1 if the buffer would overflow (nothing written then).
__device__ int gather3(const Grid& G, Cell3& C, int lane, int i, const double* ri, const int* b, int s, int s0,
                       int q0, int q1, int at) {
  const int side = 2 * s + 1;
  const int q = q0 + lane;
  int lo = 0, hi = 0, sh[3] = {0, 0, 0};
  if (q < q1) {
    const int dx = q % side - s, dy = (q / side) % side - s, dz = q / (side * side) - s;
    const int cheb = max(abs(dx), max(abs(dy), abs(dz)));
    if (cheb >= s0) {
      const int c[3] = {b[0] + dx, b[1] + dy, b[2] + dz};
      int w[3];
      for (int d = 0; d < 3; d++) {
        sh[d] = floordiv(c[d], G.nb[d]);
        w[d] = c[d] - sh[d] * G.nb[d];
      }
      const int bin = (w[2] * G.nb[1] + w[1]) * G.nb[0] + w[0];
      lo = G.bin_start[bin];
      hi = G.bin_start[bin + 1];
    }
  }
  const int cnt = hi - lo;
  int pre = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, pre, o);
    if (lane >= o) pre += y;
  }
  const int total = __shfl_sync(0xffffffffu, pre, 31);
  if (at + total > MAXC) return -1;
  int slot = at + pre - cnt;
  for (int k = lo; k < hi; k++) {
    const int j = G.bin_pts[k];
    const bool self = (j == i && sh[0] == 0 && sh[1] == 0 && sh[2] == 0);
    double d2 = 0.0;
    for (int d = 0; d < 3; d++) {
      const double x = G.pts[(size_t)j * 3 + d] + sh[d] * G.box[d] - ri[d];
      C.cx[slot][d] = x;
      d2 += x * x;
    }
    C.cd2[slot] = self ? -1.0 : d2;     // -1: the generator itself, skipped
    C.cd2f[slot] = self ? -1.0f : (float)d2;
    C.cj[slot] = j;
    for (int d = 0; d < 3; d++) C.cs[slot][d] = (signed char)sh[d];
    C.cs[slot][3] = 0;
    slot++;
  }
  __syncwarp();
  return at + total;
}

// cuts by the buffered candidates, nearest first (the near bisectors shrink
// the cell, after which most far ones miss it and are skipped unexamined);
// ties in FP32 distance keep buffer order; returns 0 or an error
__device__ int cut_buffer3(Cell3& C, int lane, int nc, double eps, float& R2) {
  for (int k = lane; k < nc; k += 32) {
    const float dk = C.cd2f[k];
    int r = 0;
    for (int u = 0; u < nc; u++) {
      const float du = C.cd2f[u];
      r += (du < dk || (du == dk && u < k)) ? 1 : 0;
    }
    C.ord[r] = (short)k;
  }
  __syncwarp();
  for (int z = 0; z < nc; z++) {
    const int k = C.ord[z];
    const float d2f = C.cd2f[k];
    // the bisector lies beyond every vertex (R2 is an FP32 upper bound)
    if (d2f < 0.0f || 0.25f * d2f >= R2 * (1.0f + 1e-5f)) continue;
    const double n[3] = {C.cx[k][0], C.cx[k][1], C.cx[k][2]};
    const int rc = cut3(C, lane, n, 0.5 * C.cd2[k], C.cj[k], C.cs[k], eps * sqrtf(d2f), R2);
    if (rc < 0) return rc;
  }
  return 0;
}

__global__ void __launch_bounds__(32 * WARPS) k_cells3(Grid G, HalfFace* hf, int* nhf, double* vol, double* com,
                                                      int* err, double thr_area) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  Cell3& C = reinterpret_cast<Cell3*>(smem)[w];
  const double hcell = fmin(G.bs[0], fmin(G.bs[1], G.bs[2]));
  const double eps = 1e-12 * hcell;
  for (int i = blockIdx.x * WARPS + w; i < G.n; i += gridDim.x * WARPS) {
    const double ri[3] = {G.pts[(size_t)i * 3], G.pts[(size_t)i * 3 + 1], G.pts[(size_t)i * 3 + 2]};
    // the initial cell: the box of the periodic domain around the generator
    if (lane < 6) {
      const int ax = lane >> 1;
      for (int d = 0; d < 3; d++) C.pn[lane][d] = (d == ax) ? ((lane & 1) ? -1.0 : 1.0) : 0.0;
      C.pn[lane][3] = 0.5 * G.box[ax];
      for (int d = 0; d < 4; d++) C.pnf[lane][d] = (float)C.pn[lane][d];
      C.pj[lane] = -1;
      for (int d = 0; d < 4; d++) C.ps[lane][d] = 0;
    }
    if (lane < 8) {
      // corner (sx, sy, sz): planes +-x, +-y, +-z, ordered so det(n_a, n_b, n_c) > 0
      const int sx = (lane & 1) ? -1 : 1, sy = (lane & 2) ? -1 : 1, sz = (lane & 4) ? -1 : 1;
      const unsigned char a = (sx > 0) ? 0 : 1, b = (sy > 0) ? 2 : 3, c = (sz > 0) ? 4 : 5;
      const bool pos = sx * sy * sz > 0;
      C.tri[lane][0] = pos ? a : b;
      C.tri[lane][1] = pos ? b : a;
      C.tri[lane][2] = c;
      C.tri[lane][3] = 1;
      const double v[3] = {sx * 0.5 * G.box[0], sy * 0.5 * G.box[1], sz * 0.5 * G.box[2]};
      set_f32(C, lane, v);
    }
    if (lane == 0) {
      C.np = 6;
      C.nt = 8;
    }
    __syncwarp();
    float R2 = 0.25f * (float)(G.box[0] * G.box[0] + G.box[1] * G.box[1] + G.box[2] * G.box[2]) * (1.0f + 1e-5f);
    int b[3];
    for (int d = 0; d < 3; d++) b[d] = bin_coord(ri[d], G.bs[d], G.nb[d]);
    const int smax = max(G.nb[0], max(G.nb[1], G.nb[2])) + 2;
    int rc = E_INCOMPLETE;
    // the first pass takes the whole 5^3 cube of bins (shells 1 and 2), so
    // the nearest candidates come first; then one shell at a time
    for (int s = 2; s <= smax && rc == E_INCOMPLETE; s++) {
      const int s0 = (s == 2) ? 0 : s;
      const int side = 2 * s + 1, nq = side * side * side;
      int nc = 0;
      int bad = 0;
      for (int q0 = 0; q0 < nq && !bad; q0 += 32) {
        const int q1 = min(nq, q0 + 32);
        int at = gather3(G, C, lane, i, ri, b, s, s0, q0, q1, nc);
        if (at < 0) {
          // buffer full: cut by what it holds, then gather again into it
          bad = cut_buffer3(C, lane, nc, eps, R2);
          nc = 0;
          if (!bad) {
            at = gather3(G, C, lane, i, ri, b, s, s0, q0, q1, 0);
            if (at < 0) bad = E_CANDIDATES;
          }
        }
        if (!bad) nc = at;
      }
      if (!bad) bad = cut_buffer3(C, lane, nc, eps, R2);
      if (bad) {
        rc = bad;
        break;
      }
      double bound = 1e300;
      for (int d = 0; d < 3; d++) {
        const double lo = (b[d] - s) * G.bs[d], hi = (b[d] + s + 1) * G.bs[d];
        bound = fmin(bound, fmin(ri[d] - lo, hi - ri[d]));
      }
      if (bound * bound >= 4.0 * (double)R2) rc = 0;
    }
    // a face of the initial box that survived: the cell is not closed
    if (rc == 0) {
      bool open = false;
      for (int t = lane; t < C.nt; t += 32)
        if (C.tri[t][3] && (C.tri[t][0] < 6 || C.tri[t][1] < 6 || C.tri[t][2] < 6)) open = true;
      if (__any_sync(0xffffffffu, open)) rc = E_OPEN;
    }
    // faces: lane per plane; the plane's vertices in cycle order, their FP64
    // positions from their three planes
    int nf = 0;
    double V = 0.0, M[3] = {0.0, 0.0, 0.0};
    if (rc == 0) {
      for (int k0 = 6; k0 < C.np; k0 += 32) {
        const int k = k0 + lane;
        double area = 0.0, fc[3] = {0.0, 0.0, 0.0};
        bool keep = false;
        if (k < C.np) {
          unsigned char nx[MAXFV], ny[MAXFV];
          short idx[MAXFV];
          int m = 0;
          for (int t = 0; t < C.nt && m < MAXFV; t++) {
            const unsigned char* tr = C.tri[t];
            if (!tr[3]) continue;
            int r = -1;
            for (int z = 0; z < 3; z++)
              if (tr[z] == k) r = z;
            if (r < 0) continue;
            nx[m] = tr[(r + 1) % 3];
            ny[m] = tr[(r + 2) % 3];
            idx[m] = (short)t;
            m++;
          }
          if (m >= 3) {
            // chain: the vertex after (k, x, y) is (k, y, .)
            short ord[MAXFV];
            int cur = 0;
            bool okc = true;
            for (int z = 0; z < m; z++) {
              ord[z] = idx[cur];
              int nxt = -1;
              for (int u = 0; u < m; u++)
                if (nx[u] == ny[cur]) nxt = u;
              if (nxt < 0) okc = false;
              cur = nxt < 0 ? 0 : nxt;
            }
            okc = okc && cur == 0;              // the cycle closes on its start
            if (okc) {
              const double* pk = C.pn[k];
              const double inv = 1.0 / sqrt(dot3(pk, pk));
              const double nk[4] = {pk[0] * inv, pk[1] * inv, pk[2] * inv, pk[3] * inv};   // unit normal, height
              double v0[3], v1[3], v2[3];
              vertex3(C, C.tri[ord[0]][0], C.tri[ord[0]][1], C.tri[ord[0]][2], v0);
              vertex3(C, C.tri[ord[1]][0], C.tri[ord[1]][1], C.tri[ord[1]][2], v2);
              for (int z = 1; z + 1 < m; z++) {
                for (int d = 0; d < 3; d++) v1[d] = v2[d];
                vertex3(C, C.tri[ord[z + 1]][0], C.tri[ord[z + 1]][1], C.tri[ord[z + 1]][2], v2);
                const double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
                const double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
                double cr[3];
                cross3(e1, e2, cr);
                const double at = 0.5 * dot3(cr, nk);
                area += at;
                for (int d = 0; d < 3; d++) fc[d] += at * (v0[d] + v1[d] + v2[d]) / 3.0;
              }
              if (area != 0.0)
                for (int d = 0; d < 3; d++) fc[d] /= area;
              area = fabs(area);
              // pyramid with apex at the generator: volume h A / 3, centroid 3/4 of the way to the face
              const double vp = nk[3] * area / 3.0;
              V += vp;
              for (int d = 0; d < 3; d++) M[d] += vp * 0.75 * fc[d];
              keep = area > thr_area;
            } else {
              rc = E_OPEN;
            }
          }
        }
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int f = nf + __popc(km & ((1u << lane) - 1u));
          if (f < MAXHF) {
            HalfFace& o = hf[(size_t)i * MAXHF + f];
            o.j = C.pj[k];
            for (int d = 0; d < 4; d++) o.s[d] = C.ps[k][d];
            o.area = area;
            for (int d = 0; d < 3; d++) o.cen[d] = fc[d];
          }
        }
        nf += __popc(km);
      }
      if (__any_sync(0xffffffffu, rc != 0)) rc = E_OPEN;
      if (nf > MAXHF) rc = E_FACES;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      V += __shfl_xor_sync(0xffffffffu, V, o);
      for (int d = 0; d < 3; d++) M[d] += __shfl_xor_sync(0xffffffffu, M[d], o);
    }
    if (lane == 0) {
      nhf[i] = rc == 0 ? nf : 0;
      vol[i] = V;
      for (int d = 0; d < 3; d++) com[(size_t)i * 3 + d] = ri[d] + (V > 0.0 ? M[d] / V : 0.0);
      if (rc != 0) atomicCAS(err, 0, rc);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------- 2D, a thread per cell
// The cell polygon as its cyclic list of lines n.x = h; vertex k is where
// line k meets line k+1.
constexpr int MAXL = 48;

struct Line2 {
  double n[2], h;
  int j;
  signed char s[2];
};

__device__ __forceinline__ void vertex2(const Line2& a, const Line2& b, double* v) {
  const double det = a.n[0] * b.n[1] - a.n[1] * b.n[0];
  v[0] = (a.h * b.n[1] - b.h * a.n[1]) / det;
  v[1] = (a.n[0] * b.h - b.n[0] * a.h) / det;
}

// cut by {x : n.x <= h}: 0 no cut, 1 cut, negative on overflow / vanished
__device__ int cut2(Line2* L, int& nl, const Line2& c, double eps, double& R2) {
  double v[MAXL][2];
  bool out[MAXL];
  int nout = 0;
  for (int k = 0; k < nl; k++) {
    vertex2(L[k], L[(k + 1) % nl], v[k]);
    out[k] = v[k][0] * c.n[0] + v[k][1] * c.n[1] - c.h > eps;
    nout += out[k] ? 1 : 0;
  }
  if (nout == 0) return 0;
  if (nout == nl) return E_VANISHED;
  // the run of outside vertices p+1..q (cyclic): lines p+2..q go, the new
  // line goes between line p+1 and line q+1
  int p = -1;
  for (int k = 0; k < nl; k++)
    if (!out[k] && out[(k + 1) % nl]) p = k;
  int q = (p + 1) % nl;
  while (out[(q + 1) % nl]) q = (q + 1) % nl;
  Line2 T[MAXL];
  int nt = 0;
  // walk from line q+1 around to line p+1, then the new line
  int k = (q + 1) % nl;
  for (;;) {
    if (nt >= MAXL - 1) return E_CAPACITY;
    T[nt++] = L[k];
    if (k == (p + 1) % nl) break;
    k = (k + 1) % nl;
  }
  T[nt++] = c;
  for (int z = 0; z < nt; z++) L[z] = T[z];
  nl = nt;
  R2 = 0.0;
  for (int z = 0; z < nl; z++) {
    double w[2];
    vertex2(L[z], L[(z + 1) % nl], w);
    R2 = fmax(R2, w[0] * w[0] + w[1] * w[1]);
  }
  return 1;
}

__global__ void k_cells2(Grid G, HalfFace* hf, int* nhf, double* vol, double* com, int* err, double thr_len) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
  const double ri[2] = {G.pts[(size_t)i * 2], G.pts[(size_t)i * 2 + 1]};
  Line2 L[MAXL];
  int nl = 4;
  const double hx = 0.5 * G.box[0], hy = 0.5 * G.box[1];
  // the box, counter-clockwise: +x, +y, -x, -y
  L[0] = {{1.0, 0.0}, hx, -1, {0, 0}};
  L[1] = {{0.0, 1.0}, hy, -1, {0, 0}};
  L[2] = {{-1.0, 0.0}, hx, -1, {0, 0}};
  L[3] = {{0.0, -1.0}, hy, -1, {0, 0}};
  double R2 = hx * hx + hy * hy;
  const double hcell = fmin(G.bs[0], G.bs[1]);
  const double eps = 1e-12 * hcell;
  const int b[2] = {bin_coord(ri[0], G.bs[0], G.nb[0]), bin_coord(ri[1], G.bs[1], G.nb[1])};
  const int smax = max(G.nb[0], G.nb[1]) + 2;
  int rc = E_INCOMPLETE;
  for (int s = 1; s <= smax && rc == E_INCOMPLETE; s++) {
    const int s0 = (s == 1) ? 0 : s;
    int bad = 0;
    for (int dy = -s; dy <= s && !bad; dy++)
      for (int dx = -s; dx <= s && !bad; dx++) {
        if (max(abs(dx), abs(dy)) < s0) continue;
        const int c[2] = {b[0] + dx, b[1] + dy};
        int sh[2], w[2];
        for (int d = 0; d < 2; d++) {
          sh[d] = floordiv(c[d], G.nb[d]);
          w[d] = c[d] - sh[d] * G.nb[d];
        }
        const int bin = w[1] * G.nb[0] + w[0];
        for (int q = G.bin_start[bin]; q < G.bin_start[bin + 1] && !bad; q++) {
          const int j = G.bin_pts[q];
          if (j == i && sh[0] == 0 && sh[1] == 0) continue;
          const double x[2] = {G.pts[(size_t)j * 2] + sh[0] * G.box[0] - ri[0],
                               G.pts[(size_t)j * 2 + 1] + sh[1] * G.box[1] - ri[1]};
          const double d2 = x[0] * x[0] + x[1] * x[1];
          if (0.25 * d2 >= R2) continue;
          const double r = sqrt(d2);
          Line2 cl;
          cl.n[0] = x[0] / r;
          cl.n[1] = x[1] / r;
          cl.h = 0.5 * r;
          cl.j = j;
          cl.s[0] = (signed char)sh[0];
          cl.s[1] = (signed char)sh[1];
          const int r2 = cut2(L, nl, cl, eps, R2);
          if (r2 < 0) bad = r2;
        }
      }
    if (bad) {
      rc = bad;
      break;
    }
    double bound = 1e300;
    for (int d = 0; d < 2; d++) {
      const double lo = (b[d] - s) * G.bs[d], hi = (b[d] + s + 1) * G.bs[d];
      bound = fmin(bound, fmin(ri[d] - lo, hi - ri[d]));
    }
    if (bound * bound >= 4.0 * R2 * (1 + 1e-12)) rc = 0;
  }
  int nf = 0;
  double V = 0.0, M[2] = {0.0, 0.0};
  if (rc == 0) {
    for (int k = 0; k < nl; k++) {
      if (L[k].j < 0) {
        rc = E_OPEN;
        break;
      }
      // edge of line k: from vertex k-1 to vertex k
      double u[2], w[2];
      vertex2(L[(k + nl - 1) % nl], L[k], u);
      vertex2(L[k], L[(k + 1) % nl], w);
      const double len = sqrt((w[0] - u[0]) * (w[0] - u[0]) + (w[1] - u[1]) * (w[1] - u[1]));
      // triangle with apex at the generator: area h len / 2, centroid 2/3 of the way to the edge midpoint
      const double at = 0.5 * L[k].h * len;
      V += at;
      M[0] += at * (2.0 / 3.0) * 0.5 * (u[0] + w[0]);
      M[1] += at * (2.0 / 3.0) * 0.5 * (u[1] + w[1]);
      if (len <= thr_len) continue;
      if (nf >= 32) {
        rc = E_CAPACITY;
        break;
      }
      HalfFace& o = hf[(size_t)i * 32 + nf];
      o.j = L[k].j;
      o.s[0] = L[k].s[0];
      o.s[1] = L[k].s[1];
      o.s[2] = 0;
      o.s[3] = 0;
      o.area = len;
      o.cen[0] = 0.5 * (u[0] + w[0]);
      o.cen[1] = 0.5 * (u[1] + w[1]);
      o.cen[2] = 0.0;
      nf++;
    }
  }
  nhf[i] = rc == 0 ? nf : 0;
  vol[i] = V;
  com[(size_t)i * 2] = ri[0] + (V > 0.0 ? M[0] / V : 0.0);
  com[(size_t)i * 2 + 1] = ri[1] + (V > 0.0 ? M[1] / V : 0.0);
  if (rc != 0) atomicCAS(err, 0, rc);
}

// --------------------------------------------------------- the face list
// A face is listed once, by the cell with the smaller index (or, for a face
// with its own periodic image, by the side whose image shift is positive).
__device__ __forceinline__ bool keep_face(int i, const HalfFace& f, int dim) {
  if (f.j != i) return f.j > i;
  for (int d = 0; d < dim; d++)
    if (f.s[d] != 0) return f.s[d] > 0;
  return false;
}

__global__ void k_keep_count(int n, int dim, int slots, const HalfFace* hf, const int* nhf, int* keep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int f = 0; f < nhf[i]; f++) c += keep_face(i, hf[(size_t)i * slots + f], dim) ? 1 : 0;
  keep[i] = c;
}

__global__ void k_emit(int n, int dim, int slots, const double* pts, const HalfFace* hf, const int* nhf,
                       const int* off, int32_t* cells, int8_t* shift, double* area, double* cen) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = off[i];
  for (int f = 0; f < nhf[i]; f++) {
    const HalfFace& h = hf[(size_t)i * slots + f];
    if (!keep_face(i, h, dim)) continue;
    cells[2 * (size_t)o] = i;
    cells[2 * (size_t)o + 1] = h.j;
    for (int d = 0; d < dim; d++) {
      shift[(size_t)o * dim + d] = h.s[d];
      cen[(size_t)o * dim + d] = pts[(size_t)i * dim + d] + h.cen[d];
    }
    area[o] = h.area;
    o++;
  }
}

// every listed face against its mirror in the neighbour's list: count the
// missing ones, the largest relative area mismatch (positive doubles order
// like their bit patterns)
__global__ void k_mirror(int n, int dim, int slots, const HalfFace* hf, const int* nhf,
                         unsigned long long* missing, unsigned long long* maxrel_bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int f = 0; f < nhf[i]; f++) {
    const HalfFace& h = hf[(size_t)i * slots + f];
    if (!keep_face(i, h, dim)) continue;
    bool found = false;
    for (int g = 0; g < nhf[h.j] && !found; g++) {
      const HalfFace& m = hf[(size_t)h.j * slots + g];
      bool same = m.j == i;
      for (int d = 0; d < dim; d++) same = same && m.s[d] == -h.s[d];
      if (same) {
        found = true;
        const double rel = fabs(m.area - h.area) / h.area;
        atomicMax(maxrel_bits, (unsigned long long)__double_as_longlong(rel));
      }
    }
    if (!found) atomicAdd(missing, 1ull);
  }
}

__global__ void k_check_range(Grid G, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
  for (int d = 0; d < G.dim; d++) {
    const double x = G.pts[(size_t)i * G.dim + d];
    if (!(x >= 0.0 && x < G.box[d])) atomicCAS(err, 0, -5);
  }
}

}  // namespace vor
}  // namespace amm

// ------------------------------------------------------------------ driver
namespace amm {
namespace vor {

// Device scratch and outputs of a build, grown on demand and kept between
// builds by a caller that tessellates repeatedly (amm_retessellate).
struct TessWork {
  int64_t cap_n = 0, cap_bins = 0, cap_hf = 0, cap_f = 0;
  int *binof = nullptr, *count = nullptr, *start = nullptr, *cursor = nullptr, *bin_pts = nullptr;
  int *err = nullptr, *nhf = nullptr, *keep = nullptr, *off = nullptr;
  HalfFace* hf = nullptr;
  unsigned long long* chk = nullptr;
  double *vol = nullptr, *com = nullptr;
  int32_t* cells = nullptr;
  int8_t* shift = nullptr;
  double *area = nullptr, *cen = nullptr;
};

TessWork* work_new() { return new TessWork(); }

void work_faces(const TessWork* w, const int32_t** cells, const int8_t** shift, const double** area,
                const double** cen) {
  *cells = w->cells;
  *shift = w->shift;
  *area = w->area;
  *cen = w->cen;
}

void work_free(TessWork* w) {
  if (!w) return;
  void* p[] = {w->binof, w->count, w->start, w->cursor, w->bin_pts, w->err, w->nhf, w->keep, w->off, w->hf,
               w->chk,   w->vol,   w->com,   w->cells,  w->shift,   w->area, w->cen};
  for (void* q : p)
    if (q) cudaFree(q);
  delete w;
}

namespace {

thread_local std::string g_tess_err;

const char* tess_msg(int rc) {
  switch (rc) {
    case -1: return "a cell has more planes or vertices than the builder holds";
    case -2: return "a cell vanished (duplicate generators)";
    case -3: return "completeness radius not reached";
    case -4: return "a cell is not closed by Voronoi faces";
    case -5: return "a generator lies outside [0, box)";
    case -6: return "a cell has more faces than the builder lists (64 in 3D, 32 in 2D)";
    case -7: return "too many generators in 32 bins of the search grid";
    default: return "tessellation failed";
  }
}

template <typename T>
cudaError_t grow(T** p, int64_t& cap, int64_t need, int64_t alloc) {
  if (need <= cap && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)std::max<int64_t>(alloc, 1));
  if (e == cudaSuccess) cap = alloc;
  return e;
}

}  // namespace

// The build: faces into w->cells/shift/area/cen (nf of them), cell volumes and
// centres into w->vol/com, half-faces per cell in w->nhf.  check: also the
// mirror test (asym, max_rel).  Returns an AMM status; the message in
// tess_last_error().
int tess_build_work(TessWork* w, int dim, int64_t n, const double* gen_d, const double* box, cudaStream_t st,
                    bool check, int64_t* nf_out, int64_t* asym, double* max_rel) {
  Grid G;
  G.dim = dim;
  G.n = (int)n;
  double vbox = 1.0;
  for (int d = 0; d < dim; d++) vbox *= box[d];
  const double hcell = std::pow(vbox / (double)n, 1.0 / dim);
  for (int d = 0; d < 3; d++) {
    if (d < dim) {
      G.nb[d] = std::max(1, (int)std::floor(box[d] / hcell + 0.5));
      G.box[d] = box[d];
      G.bs[d] = box[d] / G.nb[d];
    } else {
      G.nb[d] = 1;
      G.box[d] = 1.0;
      G.bs[d] = 1.0;
    }
  }
  const int nbins = G.nb[0] * G.nb[1] * G.nb[2];
  const int slots = dim == 3 ? MAXHF : 32;
  int rc = AMM_OK;
  auto cu = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess && rc == AMM_OK) {
      g_tess_err = std::string(where) + ": " + cudaGetErrorString(e);
      rc = AMM_ERR_CUDA;
    }
    return rc == AMM_OK;
  };
  // per-cell and per-bin scratch (sizes fixed by n, grown only)
  if (n > w->cap_n || !w->binof) {
    const int64_t m = n;
    void* p[] = {w->binof, w->bin_pts, w->nhf, w->keep, w->off, w->vol, w->com};
    for (void* q : p)
      if (q) cudaFree(q);
    w->binof = w->bin_pts = w->nhf = w->keep = w->off = nullptr;
    w->vol = w->com = nullptr;
    w->cap_n = 0;
    cu(cudaMalloc(&w->binof, sizeof(int) * m), "alloc");
    cu(cudaMalloc(&w->bin_pts, sizeof(int) * m), "alloc");
    cu(cudaMalloc(&w->nhf, sizeof(int) * m), "alloc");
    cu(cudaMalloc(&w->keep, sizeof(int) * m), "alloc");
    cu(cudaMalloc(&w->off, sizeof(int) * (m + 1)), "alloc");
    cu(cudaMalloc(&w->vol, sizeof(double) * m), "alloc");
    cu(cudaMalloc(&w->com, sizeof(double) * m * 3), "alloc");
    if (rc == AMM_OK) w->cap_n = m;
  }
  if (nbins > w->cap_bins || !w->count) {
    void* p[] = {w->count, w->start, w->cursor};
    for (void* q : p)
      if (q) cudaFree(q);
    w->count = w->start = w->cursor = nullptr;
    w->cap_bins = 0;
    cu(cudaMalloc(&w->count, sizeof(int) * nbins), "alloc");
    cu(cudaMalloc(&w->start, sizeof(int) * (nbins + 1)), "alloc");
    cu(cudaMalloc(&w->cursor, sizeof(int) * nbins), "alloc");
    if (rc == AMM_OK) w->cap_bins = nbins;
  }
  if (!w->err) cu(cudaMalloc(&w->err, sizeof(int)), "alloc");
  if (!w->chk) cu(cudaMalloc(&w->chk, sizeof(unsigned long long) * 2), "alloc");
  cu(grow(&w->hf, w->cap_hf, n * slots, n * slots), "alloc");
  if (rc != AMM_OK) return rc;
  const int nb256 = (int)((n + 255) / 256);
  G.pts = gen_d;
  cu(cudaMemsetAsync(w->count, 0, sizeof(int) * nbins, st), "memset");
  cu(cudaMemsetAsync(w->err, 0, sizeof(int), st), "memset");
  cu(cudaMemsetAsync(w->chk, 0, sizeof(unsigned long long) * 2, st), "memset");
  k_check_range<<<nb256, 256, 0, st>>>(G, w->err);
  k_bin_count<<<nb256, 256, 0, st>>>(G, w->binof, w->count);
  k_scan<<<1, 1024, 0, st>>>(w->count, w->start, nbins);
  cu(cudaMemcpyAsync(w->cursor, w->start, sizeof(int) * nbins, cudaMemcpyDeviceToDevice, st), "copy");
  k_bin_fill<<<nb256, 256, 0, st>>>(G, w->binof, w->cursor, w->bin_pts);
  k_bin_sort<<<(nbins + 255) / 256, 256, 0, st>>>(w->start, w->bin_pts, nbins);
  G.bin_start = w->start;
  G.bin_pts = w->bin_pts;
  const double thr = 1e-12 * std::pow(hcell, dim - 1);
  if (dim == 3) {
    const size_t smem = sizeof(Cell3) * WARPS;
    cu(cudaFuncSetAttribute(k_cells3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attribute");
    const int64_t blocks = std::min<int64_t>((n + WARPS - 1) / WARPS, 152 * 16);
    k_cells3<<<(int)blocks, 32 * WARPS, smem, st>>>(G, w->hf, w->nhf, w->vol, w->com, w->err, thr);
  } else {
    k_cells2<<<nb256, 256, 0, st>>>(G, w->hf, w->nhf, w->vol, w->com, w->err, thr);
  }
  k_keep_count<<<nb256, 256, 0, st>>>((int)n, dim, slots, w->hf, w->nhf, w->keep);
  k_scan<<<1, 1024, 0, st>>>(w->keep, w->off, (int)n);
  cu(cudaGetLastError(), "cells");
  int herr[2] = {0, 0};
  cu(cudaMemcpyAsync(&herr[0], w->err, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
  cu(cudaMemcpyAsync(&herr[1], w->off + n, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
  cu(cudaStreamSynchronize(st), "sync");
  if (rc != AMM_OK) return rc;
  if (herr[0] != 0) {
    g_tess_err = tess_msg(herr[0]);
    return herr[0] == -5 ? AMM_ERR_INVALID_ARG : AMM_ERR_NUMERIC;
  }
  const int64_t nf = herr[1];
  if (nf < 1) {
    g_tess_err = "no faces";
    return AMM_ERR_NUMERIC;
  }
  if (nf > w->cap_f || !w->cells) {
    const int64_t cap = nf + nf / 8;   // room for the next meshes of a moving run
    void* p[] = {w->cells, w->shift, w->area, w->cen};
    for (void* q : p)
      if (q) cudaFree(q);
    w->cells = nullptr;
    w->shift = nullptr;
    w->area = w->cen = nullptr;
    w->cap_f = 0;
    cu(cudaMalloc(&w->cells, sizeof(int32_t) * 2 * cap), "alloc");
    cu(cudaMalloc(&w->shift, (size_t)cap * 3), "alloc");
    cu(cudaMalloc(&w->area, sizeof(double) * cap), "alloc");
    cu(cudaMalloc(&w->cen, sizeof(double) * cap * 3), "alloc");
    if (rc != AMM_OK) return rc;
    w->cap_f = cap;
  }
  k_emit<<<nb256, 256, 0, st>>>((int)n, dim, slots, gen_d, w->hf, w->nhf, w->off, w->cells, w->shift, w->area,
                                w->cen);
  if (check) k_mirror<<<nb256, 256, 0, st>>>((int)n, dim, slots, w->hf, w->nhf, w->chk, w->chk + 1);
  cu(cudaGetLastError(), "faces");
  unsigned long long h[2] = {0, 0};
  if (check) cu(cudaMemcpyAsync(h, w->chk, sizeof h, cudaMemcpyDeviceToHost, st), "read");
  cu(cudaStreamSynchronize(st), "sync");
  if (rc != AMM_OK) return rc;
  *nf_out = nf;
  if (asym) *asym = (int64_t)h[0];
  if (max_rel) std::memcpy(max_rel, &h[1], sizeof(double));
  return AMM_OK;
}

const char* tess_last_error() { return g_tess_err.c_str(); }

}  // namespace vor
}  // namespace amm

// ------------------------------------------------------------------ C ABI
struct amm_tess {
  int dim = 0;
  int64_t n = 0, nf = 0;
  cudaStream_t stream = nullptr;
  amm::vor::TessWork* w = nullptr;   // owns every device array
  int64_t asym = 0;
  double max_rel = 0.0;
};

extern "C" {

const char* amm_tess_last_error(void) { return amm::vor::tess_last_error(); }

int amm_tess_build(amm_tess** out, int dim, int64_t n, const double* gen_d, const double* box, void* stream) {
  if (!out) return AMM_ERR_INVALID_ARG;
  *out = nullptr;
  if ((dim != 2 && dim != 3) || n < 2 || n > ((int64_t)1 << 30) || !gen_d || !box) return AMM_ERR_INVALID_ARG;
  for (int d = 0; d < dim; d++)
    if (!(box[d] > 0.0)) return AMM_ERR_INVALID_ARG;
  amm_tess* t = new amm_tess();
  t->dim = dim;
  t->n = n;
  t->stream = (cudaStream_t)stream;
  t->w = new amm::vor::TessWork();
  const int rc = amm::vor::tess_build_work(t->w, dim, n, gen_d, box, t->stream, true, &t->nf, &t->asym, &t->max_rel);
  if (rc != AMM_OK) {
    amm::vor::work_free(t->w);
    delete t;
    return rc;
  }
  *out = t;
  return AMM_OK;
}

int64_t amm_tess_num_faces(const amm_tess* t) { return t ? t->nf : 0; }

int amm_tess_faces(const amm_tess* t, const int32_t** cells, const int8_t** shift, const double** area,
                   const double** cen) {
  if (!t || !cells || !shift || !area || !cen) return AMM_ERR_INVALID_ARG;
  *cells = t->w->cells;
  *shift = t->w->shift;
  *area = t->w->area;
  *cen = t->w->cen;
  return AMM_OK;
}

int amm_tess_cells(const amm_tess* t, const double** vol, const double** com, const int32_t** nface) {
  if (!t || !vol || !com || !nface) return AMM_ERR_INVALID_ARG;
  *vol = t->w->vol;
  *com = t->w->com;
  *nface = t->w->nhf;
  return AMM_OK;
}

int amm_tess_check(const amm_tess* t, int64_t* asymmetric, double* max_rel) {
  if (!t || !asymmetric || !max_rel) return AMM_ERR_INVALID_ARG;
  *asymmetric = t->asym;
  *max_rel = t->max_rel;
  return AMM_OK;
}

int amm_tess_destroy(amm_tess* t) {
  if (!t) return AMM_OK;
  if (t->stream) cudaStreamSynchronize(t->stream);
  amm::vor::work_free(t->w);
  delete t;
  return AMM_OK;
}

}  // extern "C"
