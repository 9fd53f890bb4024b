// Host-side Voronoi tessellator for periodic boxes (2D and 3D).
//
// Input generator only: it turns generator positions into the face list the
// hydro update consumes (area, centroid, the two adjacent cells and the
// periodic image of the right-hand cell).  None of the hydro arithmetic lives
// here.
//
// Each cell is built as the intersection of the half-spaces bounded by the
// perpendicular bisectors between its generator and nearby generators (and
// their periodic images) -- the definition of a Voronoi cell (Sec. 2).  The
// candidate search stops once the nearest unvisited generator is farther than
// twice the largest distance from the generator to a vertex of the current
// polytope, since such a generator's bisector cannot cut the cell.  This is
// the completeness radius the paper uses for its ghost-point import (Sec. 2.4,
// the search radius versus twice the largest circumsphere radius).
//
// Faces of (numerically) zero area -- Delaunay edges whose Voronoi face
// degenerates to an edge or a point, e.g. the diagonals of an exact lattice
// (Sec. 2.3) -- are dropped.
//
// The cell volume and centre of mass are integrated directly from the
// polytope (tetrahedra about the vertex average), independently of the
// pyramid sums the hydro code derives from the face list, so the two can be
// checked against each other.
//
// Threads: std::thread over contiguous chunks of cells; the output order does
// not depend on the thread count.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct HalfFace {
  int32_t j;        // neighbour generator
  int8_t s[3];      // periodic image of the neighbour, in box lengths
  double area;      // face area (length in 2D)
  double cen[3];    // face centroid relative to the generator of this cell
};

struct CellOut {
  double vol;
  double com[3];    // centre of mass relative to the generator
  int status;       // 0 ok, else error code
};

struct Cand {
  double d2;
  int32_t j;
  int8_t s[3];
  double x[3];      // image position relative to the generator
};

inline int64_t encode_tag(int32_t j, const int8_t s[3]) {
  return (int64_t)(uint32_t)j | ((int64_t)(uint8_t)(s[0] + 128) << 32) |
         ((int64_t)(uint8_t)(s[1] + 128) << 40) | ((int64_t)(uint8_t)(s[2] + 128) << 48);
}
inline void decode_tag(int64_t t, int32_t* j, int8_t s[3]) {
  *j = (int32_t)(uint32_t)(t & 0xffffffffLL);
  s[0] = (int8_t)((int)((t >> 32) & 0xff) - 128);
  s[1] = (int8_t)((int)((t >> 40) & 0xff) - 128);
  s[2] = (int8_t)((int)((t >> 48) & 0xff) - 128);
}

// ---------------------------------------------------------------- 3D polytope
constexpr int MAXF3 = 128;
constexpr int MAXVT3 = 2048;

struct Poly3 {
  int nf = 0, nvt = 0;
  int64_t tag[MAXF3];
  int start[MAXF3], cnt[MAXF3];
  double v[MAXVT3][3];
};

inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
inline bool lex_less3(const double* a, const double* b) {
  if (a[0] != b[0]) return a[0] < b[0];
  if (a[1] != b[1]) return a[1] < b[1];
  return a[2] < b[2];
}
inline double dist2_3(const double* a, const double* b) {
  double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return dx * dx + dy * dy + dz * dz;
}

void init_box3(Poly3& P, const double* half) {
  // axis-aligned box [-half, half]; faces tagged -1 (not a Voronoi face)
  static const int F[6][4][3] = {
      {{-1, -1, -1}, {-1, 1, -1}, {-1, 1, 1}, {-1, -1, 1}},
      {{1, -1, -1}, {1, -1, 1}, {1, 1, 1}, {1, 1, -1}},
      {{-1, -1, -1}, {-1, -1, 1}, {1, -1, 1}, {1, -1, -1}},
      {{-1, 1, -1}, {1, 1, -1}, {1, 1, 1}, {-1, 1, 1}},
      {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}},
      {{-1, -1, 1}, {-1, 1, 1}, {1, 1, 1}, {1, -1, 1}}};
  P.nf = 6;
  P.nvt = 0;
  for (int f = 0; f < 6; f++) {
    P.tag[f] = -1;
    P.start[f] = P.nvt;
    P.cnt[f] = 4;
    for (int k = 0; k < 4; k++) {
      for (int d = 0; d < 3; d++) P.v[P.nvt][d] = F[f][k][d] * half[d];
      P.nvt++;
    }
  }
}

// Clip P by the half-space {p : n.p <= h}; result in Q.  Returns 0 when the
// plane does not cut P (Q untouched), 1 when Q holds the clipped polytope,
// negative on capacity overflow or a vanished cell.
int clip3(const Poly3& P, Poly3& Q, const double* n, double h, int64_t tag, double eps, double tol2,
          std::vector<double>& dist, std::vector<double>& cap) {
  dist.resize(P.nvt);
  double maxd = -1e300;
  for (int k = 0; k < P.nvt; k++) {
    dist[k] = dot3(P.v[k], n) - h;
    maxd = std::max(maxd, dist[k]);
  }
  if (maxd <= eps) return 0;
  Q.nf = 0;
  Q.nvt = 0;
  cap.clear();
  auto push_cap = [&](const double* p) { cap.push_back(p[0]); cap.push_back(p[1]); cap.push_back(p[2]); };
  for (int f = 0; f < P.nf; f++) {
    const int a = P.start[f], c = P.cnt[f];
    bool any_out = false, any_in = false;
    for (int k = 0; k < c; k++) {
      any_out |= dist[a + k] > eps;
      any_in |= dist[a + k] < -eps;
    }
    if (!any_in) {  // entirely outside or on the plane: face removed
      for (int k = 0; k < c; k++)
        if (dist[a + k] <= eps) push_cap(P.v[a + k]);
      continue;
    }
    if (Q.nf >= MAXF3) return -1;
    const int qs = Q.nvt;
    for (int k = 0; k < c; k++) {
      const int cur = a + k, nxt = a + (k + 1) % c;
      const double dc = dist[cur], dn = dist[nxt];
      const bool cur_out = dc > eps, cur_in = dc < -eps;
      const bool nxt_out = dn > eps, nxt_in = dn < -eps;
      if (!cur_out) {
        if (Q.nvt >= MAXVT3) return -1;
        std::memcpy(Q.v[Q.nvt++], P.v[cur], sizeof(double) * 3);
        if (!cur_in) push_cap(P.v[cur]);
      }
      if ((cur_in && nxt_out) || (cur_out && nxt_in)) {
        // canonical endpoint order so both faces sharing the edge get the
        // bitwise-identical intersection point
        const double *pa = P.v[cur], *pb = P.v[nxt];
        double da = dc, db = dn;
        if (lex_less3(pb, pa)) { std::swap(pa, pb); std::swap(da, db); }
        const double t = da / (da - db);
        if (Q.nvt >= MAXVT3) return -1;
        double* x = Q.v[Q.nvt++];
        for (int d = 0; d < 3; d++) x[d] = pa[d] + t * (pb[d] - pa[d]);
        push_cap(x);
      }
      (void)any_out;
    }
    // drop consecutive duplicates
    int m = Q.nvt - qs;
    int w = 0;
    for (int k = 0; k < m; k++) {
      const double* p = Q.v[qs + k];
      if (w > 0 && dist2_3(p, Q.v[qs + w - 1]) <= tol2) continue;
      if (w != k) std::memcpy(Q.v[qs + w], p, sizeof(double) * 3);
      w++;
    }
    while (w > 1 && dist2_3(Q.v[qs + w - 1], Q.v[qs]) <= tol2) w--;
    if (w >= 3) {
      Q.tag[Q.nf] = P.tag[f];
      Q.start[Q.nf] = qs;
      Q.cnt[Q.nf] = w;
      Q.nf++;
      Q.nvt = qs + w;
    } else {
      Q.nvt = qs;
    }
  }
  // the new face on the cutting plane
  const int mc = (int)cap.size() / 3;
  std::vector<int> keep;
  keep.reserve(mc);
  for (int k = 0; k < mc; k++) {
    bool dup = false;
    for (int q : keep)
      if (dist2_3(&cap[3 * k], &cap[3 * q]) <= tol2) { dup = true; break; }
    if (!dup) keep.push_back(k);
  }
  if ((int)keep.size() >= 3) {
    double cen[3] = {0, 0, 0};
    for (int q : keep)
      for (int d = 0; d < 3; d++) cen[d] += cap[3 * q + d];
    for (int d = 0; d < 3; d++) cen[d] /= (double)keep.size();
    int ax = 0;
    if (std::fabs(n[1]) < std::fabs(n[ax])) ax = 1;
    if (std::fabs(n[2]) < std::fabs(n[ax])) ax = 2;
    double e[3] = {0, 0, 0};
    e[ax] = 1;
    double u[3], w3[3];
    cross3(n, e, u);
    const double un = std::sqrt(dot3(u, u));
    for (int d = 0; d < 3; d++) u[d] /= un;
    cross3(n, u, w3);
    std::vector<std::pair<double, int>> ang;
    ang.reserve(keep.size());
    for (int q : keep) {
      double r[3] = {cap[3 * q] - cen[0], cap[3 * q + 1] - cen[1], cap[3 * q + 2] - cen[2]};
      ang.push_back({std::atan2(dot3(r, w3), dot3(r, u)), q});
    }
    std::sort(ang.begin(), ang.end());
    if (Q.nf >= MAXF3) return -1;
    const int qs = Q.nvt;
    int w = 0;
    for (auto& pr : ang) {
      const double* p = &cap[3 * pr.second];
      if (w > 0 && dist2_3(p, Q.v[qs + w - 1]) <= tol2) continue;
      if (Q.nvt >= MAXVT3) return -1;
      std::memcpy(Q.v[qs + w], p, sizeof(double) * 3);
      w++;
      Q.nvt = qs + w;
    }
    while (w > 1 && dist2_3(Q.v[qs + w - 1], Q.v[qs]) <= tol2) w--;
    if (w >= 3) {
      Q.tag[Q.nf] = tag;
      Q.start[Q.nf] = qs;
      Q.cnt[Q.nf] = w;
      Q.nf++;
      Q.nvt = qs + w;
    } else {
      Q.nvt = qs;
    }
  }
  if (Q.nf < 4) return -2;
  return 1;
}

double max_r2_3(const Poly3& P) {
  double m = 0;
  for (int k = 0; k < P.nvt; k++) m = std::max(m, dot3(P.v[k], P.v[k]));
  return m;
}

// ---------------------------------------------------------------- 2D polygon
constexpr int MAXV2 = 256;

struct Poly2 {
  int nv = 0;
  double v[MAXV2][2];
  int64_t tag[MAXV2];  // tag of the edge v[k] -> v[k+1]
};

inline double dist2_2(const double* a, const double* b) {
  double dx = a[0] - b[0], dy = a[1] - b[1];
  return dx * dx + dy * dy;
}

int clip2(const Poly2& P, Poly2& Q, const double* n, double h, int64_t tag, double eps, double tol2) {
  double dist[MAXV2];
  double maxd = -1e300;
  for (int k = 0; k < P.nv; k++) {
    dist[k] = P.v[k][0] * n[0] + P.v[k][1] * n[1] - h;
    maxd = std::max(maxd, dist[k]);
  }
  if (maxd <= eps) return 0;
  Poly2 T;
  T.nv = 0;
  auto emit = [&](const double* p, int64_t t) -> bool {
    if (T.nv >= MAXV2) return false;
    T.v[T.nv][0] = p[0];
    T.v[T.nv][1] = p[1];
    T.tag[T.nv] = t;
    T.nv++;
    return true;
  };
  for (int k = 0; k < P.nv; k++) {
    const int nx = (k + 1) % P.nv;
    const double dc = dist[k], dn = dist[nx];
    const bool cur_out = dc > eps, cur_in = dc < -eps;
    const bool nxt_out = dn > eps, nxt_in = dn < -eps;
    double X[2];
    auto isect = [&]() {
      const double *pa = P.v[k], *pb = P.v[nx];
      double da = dc, db = dn;
      if (pb[0] < pa[0] || (pb[0] == pa[0] && pb[1] < pa[1])) { std::swap(pa, pb); std::swap(da, db); }
      const double t = da / (da - db);
      X[0] = pa[0] + t * (pb[0] - pa[0]);
      X[1] = pa[1] + t * (pb[1] - pa[1]);
    };
    if (!cur_out) {
      if (nxt_out) {
        if (cur_in) {
          if (!emit(P.v[k], P.tag[k])) return -1;
          isect();
          if (!emit(X, tag)) return -1;
        } else {
          if (!emit(P.v[k], tag)) return -1;
        }
      } else {
        if (!emit(P.v[k], P.tag[k])) return -1;
      }
    } else if (nxt_in) {
      isect();
      if (!emit(X, P.tag[k])) return -1;
    }
  }
  // drop zero-length edges: keep the later vertex (its outgoing edge is real)
  Q.nv = 0;
  for (int k = 0; k < T.nv; k++) {
    const int nx = (k + 1) % T.nv;
    if (T.nv > 1 && dist2_2(T.v[k], T.v[nx]) <= tol2) continue;
    Q.v[Q.nv][0] = T.v[k][0];
    Q.v[Q.nv][1] = T.v[k][1];
    Q.tag[Q.nv] = T.tag[k];
    Q.nv++;
  }
  if (Q.nv < 3) return -2;
  return 1;
}

double max_r2_2(const Poly2& P) {
  double m = 0;
  for (int k = 0; k < P.nv; k++) m = std::max(m, P.v[k][0] * P.v[k][0] + P.v[k][1] * P.v[k][1]);
  return m;
}

// ---------------------------------------------------------------- driver
struct Grid {
  int dim;
  int64_t n;
  const double* pts;
  double box[3];
  int nb[3];
  double bs[3];
  std::vector<int64_t> bin_start;  // [nbins+1]
  std::vector<int32_t> bin_pts;
  int bin_of(const double* p, int* b) const {
    b[2] = 0;
    for (int d = 0; d < dim; d++) {
      int q = (int)std::floor(p[d] / bs[d]);
      if (q < 0) q = 0;
      if (q >= nb[d]) q = nb[d] - 1;
      b[d] = q;
    }
    return (b[2] * nb[1] + b[1]) * nb[0] + b[0];
  }
};

inline int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

// Collects candidates in bins at Chebyshev distance s0..s1 from bin b.
void gather_shell(const Grid& G, int64_t i, const int* b, int s0, int s1, std::vector<Cand>& out) {
  const double* ri = G.pts + i * G.dim;
  const int zr = (G.dim == 3) ? s1 : 0;
  for (int dz = -zr; dz <= zr; dz++)
    for (int dy = -s1; dy <= s1; dy++)
      for (int dx = -s1; dx <= s1; dx++) {
        const int cheb = std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz)));
        if (cheb < s0) continue;
        int c[3] = {b[0] + dx, b[1] + dy, b[2] + dz};
        int sh[3] = {0, 0, 0}, w[3] = {0, 0, 0};
        for (int d = 0; d < G.dim; d++) {
          sh[d] = floordiv(c[d], G.nb[d]);
          w[d] = c[d] - sh[d] * G.nb[d];
        }
        const int bin = (w[2] * G.nb[1] + w[1]) * G.nb[0] + w[0];
        for (int64_t q = G.bin_start[bin]; q < G.bin_start[bin + 1]; q++) {
          const int32_t j = G.bin_pts[q];
          if (j == i && sh[0] == 0 && sh[1] == 0 && sh[2] == 0) continue;
          Cand cd;
          cd.j = j;
          cd.d2 = 0;
          for (int d = 0; d < 3; d++) { cd.s[d] = (int8_t)sh[d]; cd.x[d] = 0; }
          for (int d = 0; d < G.dim; d++) {
            cd.x[d] = G.pts[j * G.dim + d] + sh[d] * G.box[d] - ri[d];
            cd.d2 += cd.x[d] * cd.x[d];
          }
          out.push_back(cd);
        }
      }
  std::sort(out.begin(), out.end(), [](const Cand& a, const Cand& b) {
    if (a.d2 != b.d2) return a.d2 < b.d2;
    if (a.j != b.j) return a.j < b.j;
    if (a.s[0] != b.s[0]) return a.s[0] < b.s[0];
    if (a.s[1] != b.s[1]) return a.s[1] < b.s[1];
    return a.s[2] < b.s[2];
  });
}

struct Work {
  std::vector<Poly3> p3;   // ping-pong buffers, heap-allocated (large)
  std::vector<double> dist, cap;
  std::vector<Cand> cand;
};

int build_cell3(const Grid& G, int64_t i, Work& W, std::vector<HalfFace>& faces, CellOut& co, double thr_area) {
  const double* ri = G.pts + i * 3;
  double half[3] = {0.5 * G.box[0], 0.5 * G.box[1], 0.5 * G.box[2]};
  Poly3* P = &W.p3[0];
  Poly3* Q = &W.p3[1];
  init_box3(*P, half);
  double R2 = max_r2_3(*P);
  int b[3];
  G.bin_of(ri, b);
  const double h = std::min(G.bs[0], std::min(G.bs[1], G.bs[2]));
  const double eps = 1e-12 * h, tol2 = (1e-11 * h) * (1e-11 * h);
  const int smax = std::max(G.nb[0], std::max(G.nb[1], G.nb[2])) + 2;
  bool complete = false;
  for (int s = 1; s <= smax; s++) {
    W.cand.clear();
    gather_shell(G, i, b, (s == 1) ? 0 : s, s, W.cand);
    for (const Cand& c : W.cand) {
      if (0.25 * c.d2 >= R2) break;
      const double r = std::sqrt(c.d2);
      const double n[3] = {c.x[0] / r, c.x[1] / r, c.x[2] / r};
      const int rc = clip3(*P, *Q, n, 0.5 * r, encode_tag(c.j, c.s), eps, tol2, W.dist, W.cap);
      if (rc < 0) return rc;
      if (rc == 1) {
        std::swap(P, Q);
        R2 = max_r2_3(*P);
      }
    }
    double bound = 1e300;
    for (int d = 0; d < 3; d++) {
      const double lo = (b[d] - s) * G.bs[d], hi = (b[d] + s + 1) * G.bs[d];
      bound = std::min(bound, std::min(ri[d] - lo, hi - ri[d]));
    }
    if (bound * bound >= 4.0 * R2 * (1 + 1e-12)) { complete = true; break; }
  }
  if (!complete) return -3;
  // integrate: vertex average as interior apex
  double p0[3] = {0, 0, 0};
  for (int k = 0; k < P->nvt; k++)
    for (int d = 0; d < 3; d++) p0[d] += P->v[k][d];
  for (int d = 0; d < 3; d++) p0[d] /= P->nvt;
  double vol = 0, mom[3] = {0, 0, 0};
  for (int f = 0; f < P->nf; f++) {
    if (P->tag[f] == -1) return -4;  // a face of the initial box survived
    const int a = P->start[f], c = P->cnt[f];
    // face area and centroid: fan about the first vertex, signed along the
    // Newell normal of the polygon
    double N[3] = {0, 0, 0};
    for (int k = 0; k < c; k++) {
      const double* u = P->v[a + k];
      const double* w = P->v[a + (k + 1) % c];
      N[0] += (u[1] - w[1]) * (u[2] + w[2]);
      N[1] += (u[2] - w[2]) * (u[0] + w[0]);
      N[2] += (u[0] - w[0]) * (u[1] + w[1]);
    }
    const double nn = std::sqrt(dot3(N, N));
    double area = 0, fc[3] = {0, 0, 0}, fv = 0, fm[3] = {0, 0, 0};
    if (nn > 0) {
      for (int d = 0; d < 3; d++) N[d] /= nn;
      const double* v0 = P->v[a];
      for (int k = 1; k + 1 < c; k++) {
        const double* v1 = P->v[a + k];
        const double* v2 = P->v[a + k + 1];
        double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
        double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
        double cr[3];
        cross3(e1, e2, cr);
        const double at = 0.5 * dot3(cr, N);
        area += at;
        for (int d = 0; d < 3; d++) fc[d] += at * (v0[d] + v1[d] + v2[d]) / 3.0;
        double q0[3] = {v0[0] - p0[0], v0[1] - p0[1], v0[2] - p0[2]};
        double q1[3] = {v1[0] - p0[0], v1[1] - p0[1], v1[2] - p0[2]};
        double q2[3] = {v2[0] - p0[0], v2[1] - p0[1], v2[2] - p0[2]};
        double c12[3];
        cross3(q1, q2, c12);
        const double vt = dot3(q0, c12) / 6.0;
        fv += vt;
        for (int d = 0; d < 3; d++) fm[d] += vt * (p0[d] + v0[d] + v1[d] + v2[d]) / 4.0;
      }
    }
    if (area != 0)
      for (int d = 0; d < 3; d++) fc[d] /= area;
    const double sgn = (fv < 0) ? -1.0 : 1.0;
    vol += sgn * fv;
    for (int d = 0; d < 3; d++) mom[d] += sgn * fm[d];
    area = std::fabs(area);
    if (area <= thr_area) continue;
    HalfFace hf;
    decode_tag(P->tag[f], &hf.j, hf.s);
    hf.area = area;
    for (int d = 0; d < 3; d++) hf.cen[d] = fc[d];
    faces.push_back(hf);
  }
  co.vol = vol;
  for (int d = 0; d < 3; d++) co.com[d] = mom[d] / vol;
  return 0;
}

int build_cell2(const Grid& G, int64_t i, Work& W, std::vector<HalfFace>& faces, CellOut& co, double thr_area) {
  const double* ri = G.pts + i * 2;
  Poly2 A, B;
  Poly2* P = &A;
  Poly2* Q = &B;
  const double hx = 0.5 * G.box[0], hy = 0.5 * G.box[1];
  P->nv = 4;
  const double sq[4][2] = {{-hx, -hy}, {hx, -hy}, {hx, hy}, {-hx, hy}};
  for (int k = 0; k < 4; k++) {
    P->v[k][0] = sq[k][0];
    P->v[k][1] = sq[k][1];
    P->tag[k] = -1;
  }
  double R2 = max_r2_2(*P);
  int b[3];
  G.bin_of(ri, b);
  const double h = std::min(G.bs[0], G.bs[1]);
  const double eps = 1e-12 * h, tol2 = (1e-11 * h) * (1e-11 * h);
  const int smax = std::max(G.nb[0], G.nb[1]) + 2;
  bool complete = false;
  for (int s = 1; s <= smax; s++) {
    W.cand.clear();
    gather_shell(G, i, b, (s == 1) ? 0 : s, s, W.cand);
    for (const Cand& c : W.cand) {
      if (0.25 * c.d2 >= R2) break;
      const double r = std::sqrt(c.d2);
      const double n[2] = {c.x[0] / r, c.x[1] / r};
      const int rc = clip2(*P, *Q, n, 0.5 * r, encode_tag(c.j, c.s), eps, tol2);
      if (rc < 0) return rc;
      if (rc == 1) {
        std::swap(P, Q);
        R2 = max_r2_2(*P);
      }
    }
    double bound = 1e300;
    for (int d = 0; d < 2; d++) {
      const double lo = (b[d] - s) * G.bs[d], hi = (b[d] + s + 1) * G.bs[d];
      bound = std::min(bound, std::min(ri[d] - lo, hi - ri[d]));
    }
    if (bound * bound >= 4.0 * R2 * (1 + 1e-12)) { complete = true; break; }
  }
  if (!complete) return -3;
  double p0[2] = {0, 0};
  for (int k = 0; k < P->nv; k++) { p0[0] += P->v[k][0]; p0[1] += P->v[k][1]; }
  p0[0] /= P->nv;
  p0[1] /= P->nv;
  double area = 0, mom[2] = {0, 0};
  for (int k = 0; k < P->nv; k++) {
    const double* u = P->v[k];
    const double* w = P->v[(k + 1) % P->nv];
    if (P->tag[k] == -1) return -4;
    const double at = 0.5 * ((u[0] - p0[0]) * (w[1] - p0[1]) - (u[1] - p0[1]) * (w[0] - p0[0]));
    area += at;
    mom[0] += at * (p0[0] + u[0] + w[0]) / 3.0;
    mom[1] += at * (p0[1] + u[1] + w[1]) / 3.0;
    const double len = std::sqrt(dist2_2(u, w));
    if (len <= thr_area) continue;
    HalfFace hf;
    decode_tag(P->tag[k], &hf.j, hf.s);
    hf.area = len;
    hf.cen[0] = 0.5 * (u[0] + w[0]);
    hf.cen[1] = 0.5 * (u[1] + w[1]);
    hf.cen[2] = 0;
    faces.push_back(hf);
  }
  co.vol = std::fabs(area);
  co.com[0] = mom[0] / area;
  co.com[1] = mom[1] / area;
  co.com[2] = 0;
  return 0;
}

inline bool shift_positive(const int8_t* s) {
  if (s[0] != 0) return s[0] > 0;
  if (s[1] != 0) return s[1] > 0;
  return s[2] > 0;
}

}  // namespace

struct tess_result {
  int dim;
  int64_t n;
  std::vector<int32_t> cells;   // [F][2]
  std::vector<int8_t> shift;    // [F][dim]
  std::vector<double> area;     // [F]
  std::vector<double> cen;      // [F][dim], absolute, in the frame of the left cell
  std::vector<double> vol;      // [n]
  std::vector<double> com;      // [n][dim], absolute
  std::vector<int32_t> nface;   // [n] faces (both sides) per cell
  int64_t asym = 0;             // faces whose mirror was not found by the other cell
  double max_asym_rel = 0;      // largest relative area mismatch between the two sides
};

extern "C" {

// Returns 0 on success.  Error codes: -1 capacity overflow, -2 vanished cell
// (duplicate generators), -3 completeness not reached, -4 cell not closed,
// -5 bad arguments.
int tess_build(int dim, int64_t n, const double* pts, const double* box, int nthreads, tess_result** out) {
  *out = nullptr;
  if ((dim != 2 && dim != 3) || n < 2 || !pts || !box) return -5;
  Grid G;
  G.dim = dim;
  G.n = n;
  G.pts = pts;
  double vbox = 1;
  for (int d = 0; d < dim; d++) {
    G.box[d] = box[d];
    vbox *= box[d];
  }
  const double hcell = std::pow(vbox / (double)n, 1.0 / dim);
  for (int d = 0; d < 3; d++) {
    if (d < dim) {
      G.nb[d] = std::max(1, (int)std::floor(box[d] / hcell + 0.5));
      G.bs[d] = box[d] / G.nb[d];
    } else {
      G.nb[d] = 1;
      G.bs[d] = 1;
      G.box[d] = 1;
    }
  }
  for (int64_t i = 0; i < n; i++)
    for (int d = 0; d < dim; d++)
      if (!(pts[i * dim + d] >= 0 && pts[i * dim + d] < box[d])) return -5;
  const int64_t nbins = (int64_t)G.nb[0] * G.nb[1] * G.nb[2];
  G.bin_start.assign(nbins + 1, 0);
  std::vector<int32_t> binof(n);
  for (int64_t i = 0; i < n; i++) {
    int b[3];
    binof[i] = G.bin_of(pts + i * dim, b);
    G.bin_start[binof[i] + 1]++;
  }
  for (int64_t k = 0; k < nbins; k++) G.bin_start[k + 1] += G.bin_start[k];
  G.bin_pts.resize(n);
  {
    std::vector<int64_t> fill(G.bin_start.begin(), G.bin_start.end() - 1);
    for (int64_t i = 0; i < n; i++) G.bin_pts[fill[binof[i]]++] = (int32_t)i;
  }
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  const int64_t chunk = 2048;
  const int64_t nchunks = (n + chunk - 1) / chunk;
  std::vector<std::vector<HalfFace>> cfaces(nchunks);
  std::vector<std::vector<int32_t>> ccount(nchunks);
  std::vector<CellOut> cells(n);
  std::atomic<int64_t> next(0);
  std::atomic<int> err(0);
  const double thr_area = 1e-12 * std::pow(hcell, dim - 1);
  auto worker = [&]() {
    Work W;
    W.p3.resize(dim == 3 ? 2 : 0);
    for (;;) {
      const int64_t c = next.fetch_add(1);
      if (c >= nchunks || err.load() != 0) break;
      const int64_t i0 = c * chunk, i1 = std::min(n, i0 + chunk);
      std::vector<HalfFace>& hf = cfaces[c];
      std::vector<int32_t>& cnt = ccount[c];
      cnt.resize(i1 - i0);
      for (int64_t i = i0; i < i1; i++) {
        const size_t before = hf.size();
        const int rc = (dim == 3) ? build_cell3(G, i, W, hf, cells[i], thr_area)
                                  : build_cell2(G, i, W, hf, cells[i], thr_area);
        if (rc != 0) {
          int z = 0;
          err.compare_exchange_strong(z, rc);
          break;
        }
        cnt[i - i0] = (int32_t)(hf.size() - before);
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; t++) th.emplace_back(worker);
  for (auto& t : th) t.join();
  if (err.load() != 0) return err.load();

  // per-cell half-face offsets
  std::vector<int64_t> hoff(n + 1, 0);
  for (int64_t c = 0; c < nchunks; c++)
    for (size_t k = 0; k < ccount[c].size(); k++) hoff[c * chunk + k + 1] = ccount[c][k];
  for (int64_t i = 0; i < n; i++) hoff[i + 1] += hoff[i];
  std::vector<HalfFace> all(hoff[n]);
  {
    size_t w = 0;
    for (int64_t c = 0; c < nchunks; c++)
      for (auto& f : cfaces[c]) all[w++] = f;
    cfaces.clear();
  }
  tess_result* R = new tess_result();
  R->dim = dim;
  R->n = n;
  R->vol.resize(n);
  R->com.resize(n * dim);
  R->nface.resize(n);
  for (int64_t i = 0; i < n; i++) {
    R->vol[i] = cells[i].vol;
    for (int d = 0; d < dim; d++) R->com[i * dim + d] = pts[i * dim + d] + cells[i].com[d];
    R->nface[i] = (int32_t)(hoff[i + 1] - hoff[i]);
  }
  int64_t asym = 0;
  double maxrel = 0;
  for (int64_t i = 0; i < n; i++) {
    for (int64_t q = hoff[i]; q < hoff[i + 1]; q++) {
      const HalfFace& f = all[q];
      const bool keep = (f.j > i) || (f.j == i && shift_positive(f.s));
      if (!keep) continue;
      R->cells.push_back((int32_t)i);
      R->cells.push_back(f.j);
      for (int d = 0; d < dim; d++) R->shift.push_back(f.s[d]);
      R->area.push_back(f.area);
      for (int d = 0; d < dim; d++) R->cen.push_back(pts[i * dim + d] + f.cen[d]);
      // mirror on the other side
      bool found = false;
      for (int64_t r = hoff[f.j]; r < hoff[f.j + 1]; r++) {
        const HalfFace& g = all[r];
        if (g.j == i && g.s[0] == -f.s[0] && g.s[1] == -f.s[1] && g.s[2] == -f.s[2]) {
          found = true;
          maxrel = std::max(maxrel, std::fabs(g.area - f.area) / f.area);
          break;
        }
      }
      if (!found) asym++;
    }
  }
  R->asym = asym;
  R->max_asym_rel = maxrel;
  *out = R;
  return 0;
}

int64_t tess_num_faces(const tess_result* R) { return (int64_t)R->area.size(); }
int64_t tess_num_asymmetric(const tess_result* R) { return R->asym; }
double tess_max_asym_rel(const tess_result* R) { return R->max_asym_rel; }

void tess_get_faces(const tess_result* R, int32_t* cells, int8_t* shift, double* area, double* cen) {
  std::memcpy(cells, R->cells.data(), R->cells.size() * sizeof(int32_t));
  std::memcpy(shift, R->shift.data(), R->shift.size() * sizeof(int8_t));
  std::memcpy(area, R->area.data(), R->area.size() * sizeof(double));
  std::memcpy(cen, R->cen.data(), R->cen.size() * sizeof(double));
}

void tess_get_cells(const tess_result* R, double* vol, double* com, int32_t* nface) {
  std::memcpy(vol, R->vol.data(), R->vol.size() * sizeof(double));
  std::memcpy(com, R->com.data(), R->com.size() * sizeof(double));
  std::memcpy(nface, R->nface.data(), R->nface.size() * sizeof(int32_t));
}

void tess_free(tess_result* R) { delete R; }

}  // extern "C"
