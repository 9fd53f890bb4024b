/*
 * amm_oracle.c -- plain, slow, FP64 CPU oracle of one moving-mesh
 * MUSCL-Hancock update on a given Voronoi tessellation (Springel 2010,
 * "E pur si muove", Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code with the CUDA
 * path and must never be called by it.
 *
 * Every function follows one passage of the paper, step by step, in its order
 * and notation; nothing is blocked, fused or reordered.  Build with
 * -O2 -ffp-contract=off.
 *
 * Conventions.  Face k joins cell L = cells[2k] and cell R = cells[2k+1]; the
 * right cell's generator is taken in the periodic image
 * r_R + shift[k] * box, and the face centroid cen[k] is given in the left
 * cell's frame.  Per-cell arrays: Q = (m, p_1..p_D, E), W = (rho, v_1..v_D, P),
 * gradients grad[i][var][axis] with var over the D+2 primitives.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV_MAX 6 /* D + 2 primitives for D <= 3, and the entropic function */

/* ------------------------------------------------------------ host threads
 * The per-cell and per-face loops have independent iterations.  They may run
 * on several host threads: [0, n) is cut into contiguous chunks, one per
 * thread, and every element runs the same code whatever the thread count.
 * The only results shared between elements are integer counters (summed per
 * chunk, then over the chunks) and the time-step minimum (taken afterwards
 * over the per-cell values), so the output does not depend on the thread
 * count.  One thread by default. */
typedef void (*elem_fn)(const void* args, long i, int64_t* counters);

typedef struct {
  elem_fn fn;
  const void* args;
  long lo, hi;
  int64_t cnt[4];
} chunk_job;

static int ora_threads = 1;

void ora_set_threads(int t) { ora_threads = t < 1 ? 1 : (t > 256 ? 256 : t); }
int ora_get_threads(void) { return ora_threads; }

static void* run_chunk(void* p) {
  chunk_job* j = (chunk_job*)p;
  for (long i = j->lo; i < j->hi; i++) j->fn(j->args, i, j->cnt);
  return NULL;
}

/* fn(args, i, counters) for i in [0, n); counters (4 slots, may be NULL)
 * receive the sums of the per-chunk counters */
static void par_for(long n, elem_fn fn, const void* args, int64_t* counters) {
  int T = ora_threads;
  if ((long)T > n) T = n > 0 ? (int)n : 1;
  chunk_job* jobs = (chunk_job*)calloc((size_t)T, sizeof(chunk_job));
  pthread_t* th = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
  char* started = (char*)calloc((size_t)T, 1);
  for (int c = 0; c < T; c++) {
    jobs[c].fn = fn;
    jobs[c].args = args;
    jobs[c].lo = n * c / T;
    jobs[c].hi = n * (c + 1) / T;
  }
  for (int c = 1; c < T; c++) started[c] = pthread_create(&th[c], NULL, run_chunk, &jobs[c]) == 0;
  run_chunk(&jobs[0]);
  for (int c = 1; c < T; c++) {
    if (started[c])
      pthread_join(th[c], NULL);
    else
      run_chunk(&jobs[c]);
  }
  if (counters)
    for (int c = 0; c < T; c++)
      for (int q = 0; q < 4; q++) counters[q] += jobs[c].cnt[q];
  free(jobs);
  free(th);
  free(started);
}

/* ------------------------------------------------------------------ helpers */

static void face_positions(int dim, long k, const double* gen, const int32_t* cells, const int8_t* shift,
                           const double* box, double* rL, double* rR) {
  const int L = cells[2 * k], R = cells[2 * k + 1];
  for (int d = 0; d < dim; d++) {
    rL[d] = gen[(long)L * dim + d];
    rR[d] = gen[(long)R * dim + d] + shift[k * dim + d] * box[d];
  }
}

/* Cell -> (face, side) incidence lists in face order; side 0 = left, 1 = right. */
typedef struct {
  long* off;
  long* face;
  int* side;
} incidence;

static incidence build_incidence(long n, long nf, const int32_t* cells) {
  incidence I;
  I.off = (long*)calloc((size_t)n + 1, sizeof(long));
  I.face = (long*)malloc(sizeof(long) * (size_t)(2 * nf + 1));
  I.side = (int*)malloc(sizeof(int) * (size_t)(2 * nf + 1));
  for (long k = 0; k < nf; k++) {
    I.off[cells[2 * k] + 1]++;
    I.off[cells[2 * k + 1] + 1]++;
  }
  for (long i = 0; i < n; i++) I.off[i + 1] += I.off[i];
  long* fill = (long*)malloc(sizeof(long) * (size_t)(n + 1));
  memcpy(fill, I.off, sizeof(long) * (size_t)(n + 1));
  for (long k = 0; k < nf; k++) {
    for (int s = 0; s < 2; s++) {
      const long c = cells[2 * k + s];
      I.face[fill[c]] = k;
      I.side[fill[c]] = s;
      fill[c]++;
    }
  }
  free(fill);
  return I;
}

static void free_incidence(incidence* I) {
  free(I->off);
  free(I->face);
  free(I->side);
}

/* For cell i seen through face k from `side`: its own generator r_i, the
 * neighbour's generator r_j and the face centroid f, all in cell i's frame. */
static void incidence_geometry(int dim, long k, int side, const double* gen, const int32_t* cells,
                               const int8_t* shift, const double* cen, const double* box, double* ri, double* rj,
                               double* f) {
  double rL[3], rR[3];
  face_positions(dim, k, gen, cells, shift, box, rL, rR);
  for (int d = 0; d < dim; d++) {
    if (side == 0) {
      ri[d] = rL[d];
      rj[d] = rR[d];
      f[d] = cen[k * dim + d];
    } else {
      const double sh = shift[k * dim + d] * box[d];
      ri[d] = rR[d] - sh; /* = generator of R in its own frame */
      rj[d] = rL[d] - sh;
      f[d] = cen[k * dim + d] - sh;
    }
  }
}

/* ---------------------------------------------------- A0: volumes, centroids
 * Sec. 2.3: a cell's volume is the sum of the pyramids spanned by its faces
 * and its generator; the pyramid over face k has height |r_R - r_L| / 2.
 * The centre of mass is the volume-weighted mean of the pyramid centroids,
 * which sit a fraction D/(D+1) of the way from the apex to the base centroid.
 * Returns 0, or -1 if a cell has non-positive volume. */
int ora_geometry(int dim, long n, const double* gen, long nf, const int32_t* cells, const int8_t* shift,
                 const double* area, const double* cen, const double* box, double* V, double* s) {
  double* mom = (double*)calloc((size_t)n * dim, sizeof(double));
  for (long i = 0; i < n; i++) V[i] = 0.0;
  for (long k = 0; k < nf; k++) {
    const int L = cells[2 * k], R = cells[2 * k + 1];
    double rL[3], rR[3];
    face_positions(dim, k, gen, cells, shift, box, rL, rR);
    double sep = 0.0;
    for (int d = 0; d < dim; d++) sep += (rR[d] - rL[d]) * (rR[d] - rL[d]);
    sep = sqrt(sep);
    const double vpyr = area[k] * (0.5 * sep) / dim;
    const double frac = (double)dim / (double)(dim + 1);
    V[L] += vpyr;
    V[R] += vpyr;
    for (int d = 0; d < dim; d++) {
      const double f = cen[k * dim + d];
      /* left pyramid, in L's frame */
      mom[(long)L * dim + d] += vpyr * (rL[d] + frac * (f - rL[d]));
      /* right pyramid, apex at the image of R; shifted back into R's frame */
      const double sh = shift[k * dim + d] * box[d];
      mom[(long)R * dim + d] += vpyr * (rR[d] + frac * (f - rR[d]) - sh);
    }
  }
  int bad = 0;
  for (long i = 0; i < n; i++) {
    if (!(V[i] > 0.0)) bad = 1;
    for (int d = 0; d < dim; d++) s[i * dim + d] = mom[i * dim + d] / V[i];
  }
  free(mom);
  return bad ? -1 : 0;
}

/* ------------------------------------------------ A1: conserved -> primitive
 * Sec. 3, step 2 and the equation of state P = (gamma-1) rho u:
 * rho = m/V, v = p/m, P = (gamma-1) (E/V - rho |v|^2 / 2). */
typedef struct {
  int dim;
  const double *Q, *V;
  double gamma;
  double* W;
} prim_args;

static void prim_cell(const void* a, long i, int64_t* counters) {
  (void)counters;
  const prim_args* A = (const prim_args*)a;
  const int dim = A->dim;
  const double *Q = A->Q, *V = A->V;
  const double gamma = A->gamma;
  double* W = A->W;
  const int nv = dim + 2;
  {
    const double m = Q[i * nv];
    const double rho = m / V[i];
    double v2 = 0.0;
    W[i * nv] = rho;
    for (int d = 0; d < dim; d++) {
      const double v = Q[i * nv + 1 + d] / m;
      W[i * nv + 1 + d] = v;
      v2 += v * v;
    }
    const double E = Q[i * nv + dim + 1];
    W[i * nv + dim + 1] = (gamma - 1.0) * (E / V[i] - 0.5 * rho * v2);
  }
}

void ora_primitives(int dim, long n, const double* Q, const double* V, double gamma, double* W) {
  const prim_args A = {dim, Q, V, gamma, W};
  par_for(n, prim_cell, &A, NULL);
}

/* ---------------------------------------------- A2 + A3: gradients, limiter
 * Gradient, eq. (eqngrad2), Sec. 3.1:
 *   <grad phi>_i = (1/V_i) sum_j A_ij ( [phi_j - phi_i] c_ij / r_ij
 *                                       - (phi_i + phi_j)/2 * r_ij_vec / r_ij )
 * with r_ij_vec = r_i - r_j and c_ij = f_ij - (r_i + r_j)/2.
 * Limiter, Sec. 3.1 (Barth-Jespersen form): per primitive variable
 * alpha_i = min(1, min_j psi_ij), psi_ij = (phi_max - phi_i)/dphi for dphi>0,
 * (phi_min - phi_i)/dphi for dphi<0, 1 for dphi=0, dphi = grad . (f_ij - s_i);
 * phi_max/phi_min over the neighbours and the cell itself (the paper's second
 * "max" is read as "min").  grad: [n][dim+2][dim]. */
typedef struct {
  int dim;
  const double *W, *gen, *V, *s;
  const int32_t* cells;
  const int8_t* shift;
  const double *area, *cen, *box;
  int limit;
  double* grad;
  const incidence* I;
  int nv;  /* variables per cell in W and grad */
} grad_args;

static void grad_cell(const void* a, long i, int64_t* counters) {
  (void)counters;
  const grad_args* A = (const grad_args*)a;
  const int dim = A->dim;
  const double *W = A->W, *gen = A->gen, *V = A->V, *s = A->s;
  const int32_t* cells = A->cells;
  const int8_t* shift = A->shift;
  const double *area = A->area, *cen = A->cen, *box = A->box;
  const int limit = A->limit;
  double* grad = A->grad;
  const incidence I = *A->I;
  const int nv = A->nv;
  {
    double g[NV_MAX][3];
    for (int v = 0; v < nv; v++)
      for (int d = 0; d < 3; d++) g[v][d] = 0.0;
    for (long q = I.off[i]; q < I.off[i + 1]; q++) {
      const long k = I.face[q];
      const int side = I.side[q];
      const long j = cells[2 * k + (1 - side)];
      double ri[3], rj[3], f[3];
      incidence_geometry(dim, k, side, gen, cells, shift, cen, box, ri, rj, f);
      double rij[3], c[3], r = 0.0;
      for (int d = 0; d < dim; d++) {
        rij[d] = ri[d] - rj[d];
        c[d] = f[d] - 0.5 * (ri[d] + rj[d]);
        r += rij[d] * rij[d];
      }
      r = sqrt(r);
      for (int v = 0; v < nv; v++) {
        const double phi_i = W[i * nv + v], phi_j = W[j * nv + v];
        for (int d = 0; d < dim; d++)
          g[v][d] += area[k] * ((phi_j - phi_i) * c[d] / r - 0.5 * (phi_i + phi_j) * rij[d] / r);
      }
    }
    for (int v = 0; v < nv; v++)
      for (int d = 0; d < dim; d++) g[v][d] /= V[i];

    if (limit) {
      for (int v = 0; v < nv; v++) {
        const double phi_i = W[i * nv + v];
        double phi_max = phi_i, phi_min = phi_i;
        for (long q = I.off[i]; q < I.off[i + 1]; q++) {
          const long k = I.face[q];
          const long j = cells[2 * k + (1 - I.side[q])];
          const double phi_j = W[j * nv + v];
          if (phi_j > phi_max) phi_max = phi_j;
          if (phi_j < phi_min) phi_min = phi_j;
        }
        double alpha = 1.0;
        for (long q = I.off[i]; q < I.off[i + 1]; q++) {
          const long k = I.face[q];
          double ri[3], rj[3], f[3];
          incidence_geometry(dim, k, I.side[q], gen, cells, shift, cen, box, ri, rj, f);
          double dphi = 0.0;
          for (int d = 0; d < dim; d++) dphi += g[v][d] * (f[d] - s[i * dim + d]);
          double psi;
          if (dphi > 0.0)
            psi = (phi_max - phi_i) / dphi;
          else if (dphi < 0.0)
            psi = (phi_min - phi_i) / dphi;
          else
            psi = 1.0;
          if (psi < alpha) alpha = psi;
        }
        for (int d = 0; d < dim; d++) g[v][d] *= alpha;
      }
    }
    for (int v = 0; v < nv; v++)
      for (int d = 0; d < dim; d++) grad[(i * nv + v) * dim + d] = g[v][d];
  }
}

void ora_gradients(int dim, long n, const double* W, const double* gen, const double* V, const double* s, long nf,
                   const int32_t* cells, const int8_t* shift, const double* area, const double* cen,
                   const double* box, int limit, double* grad) {
  incidence I = build_incidence(n, nf, cells);
  const grad_args A = {dim, W, gen, V, s, cells, shift, area, cen, box, limit, grad, &I, dim + 2};
  par_for(n, grad_cell, &A, NULL);
  free_incidence(&I);
}

/* the same for nvar variables per cell (W [n][nvar], grad [n][nvar][dim]) */
static void gradients_nvar(int dim, long n, int nvar, const double* W, const double* gen, const double* V,
                           const double* s, long nf, const int32_t* cells, const int8_t* shift, const double* area,
                           const double* cen, const double* box, int limit, double* grad) {
  incidence I = build_incidence(n, nf, cells);
  const grad_args A = {dim, W, gen, V, s, cells, shift, area, cen, box, limit, grad, &I, nvar};
  par_for(n, grad_cell, &A, NULL);
  free_incidence(&I);
}

/* ---------------------------------------------------------- A4: CFL step
 * Eq. (EqnTiStep), Sec. 7.1: dt_i = C_CFL R_i / (c_i + |v_i - w_i|), with
 * R_i = (3 V_i / 4 pi)^(1/3) in 3D, (V_i / pi)^(1/2) in 2D, c_i = sqrt(gamma
 * P/rho); the global step is the minimum over cells.  wmesh may be NULL (0). */
typedef struct {
  int dim;
  const double *W, *V, *wmesh;
  double gamma, cfl;
  double* dt_cell;
} ts_args;

static void ts_cell(const void* a, long i, int64_t* counters) {
  (void)counters;
  const ts_args* A = (const ts_args*)a;
  const int dim = A->dim;
  const double *W = A->W, *V = A->V, *wmesh = A->wmesh;
  const double gamma = A->gamma, cfl = A->cfl;
  const int nv = dim + 2;
  {
    const double rho = W[i * nv], P = W[i * nv + dim + 1];
    const double R = (dim == 3) ? cbrt(3.0 * V[i] / (4.0 * M_PI)) : sqrt(V[i] / M_PI);
    const double c = sqrt(gamma * P / rho);
    double vr = 0.0;
    for (int d = 0; d < dim; d++) {
      const double dv = W[i * nv + 1 + d] - (wmesh ? wmesh[i * dim + d] : 0.0);
      vr += dv * dv;
    }
    const double dt = cfl * R / (c + sqrt(vr));
    A->dt_cell[i] = dt;
  }
}

double ora_timestep(int dim, long n, const double* W, const double* V, const double* wmesh, double gamma,
                    double cfl, double* dt_cell) {
  double* dtc = dt_cell ? dt_cell : (double*)malloc(sizeof(double) * (size_t)(n + 1));
  const ts_args A = {dim, W, V, wmesh, gamma, cfl, dtc};
  par_for(n, ts_cell, &A, NULL);
  double dtmin = INFINITY;
  for (long i = 0; i < n; i++)
    if (dtc[i] < dtmin) dtmin = dtc[i];
  if (!dt_cell) free(dtc);
  return dtmin;
}

/* ------------------------------------------------ A7: exact Riemann solver
 * Sec. 3.3 names an exact solver for the ideal gas with an extension for
 * vacuum states.  Written here from the gas dynamics of the 1D Riemann
 * problem: the star pressure p* is the root of
 *   f(p) = f_L(p) + f_R(p) + (u_R - u_L),
 *   f_K(p) = (p - p_K) sqrt(A_K / (p + B_K))              (shock, p > p_K)
 *          = 2 c_K/(gamma-1) ((p/p_K)^((gamma-1)/(2gamma)) - 1)   (rarefaction)
 *   A_K = 2/((gamma+1) rho_K), B_K = (gamma-1)/(gamma+1) p_K,
 * found by Newton from the adaptive primitive-variable / two-rarefaction /
 * two-shock guess, to the relative change 2|dp|/(p_new+p_old) < tol (or to a
 * residual f(p) at the rounding level of its terms); then
 * u* = (u_L+u_R)/2 + (f_R(p*) - f_L(p*))/2 and the self-similar solution is
 * sampled at x/t = 0.  Vacuum: a vacuum side, or vacuum generated between two
 * rarefactions when 2(c_L+c_R)/(gamma-1) <= u_R - u_L; the sampled state in
 * vacuum is rho = P = 0.
 *
 * in: (rho, u, p) per side.  out: rho, u, p at x/t=0, p*, u*, side (0 left of
 * the contact, 1 right; decides the upwind transverse velocity).
 * Returns 0 ok, 1 vacuum involved, -1 Newton did not converge in maxit. */

static double pfun(double p, double rhoK, double pK, double cK, double g, double* dfdp) {
  if (p > pK) {
    const double A = 2.0 / ((g + 1.0) * rhoK);
    const double B = (g - 1.0) / (g + 1.0) * pK;
    const double q = sqrt(A / (p + B));
    *dfdp = q * (1.0 - 0.5 * (p - pK) / (p + B));
    return (p - pK) * q;
  }
  const double pr = p / pK;
  *dfdp = pow(pr, -(g + 1.0) / (2.0 * g)) / (rhoK * cK);
  return 2.0 * cK / (g - 1.0) * (pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
}

/* state inside a rarefaction fan (left-facing if dir = -1, right-facing +1)
 * at x/t = S, from the isentropic relations and the Riemann invariant */
static void fan_state(double g, double rhoK, double uK, double pK, double cK, int dir, double S, double* rho,
                      double* u, double* p) {
  double c;
  if (dir < 0) { /* left wave: u + 2c/(g-1) constant, S = u - c */
    c = 2.0 / (g + 1.0) * cK + (g - 1.0) / (g + 1.0) * (uK - S);
    *u = S + c;
  } else { /* right wave: u - 2c/(g-1) constant, S = u + c */
    c = 2.0 / (g + 1.0) * cK - (g - 1.0) / (g + 1.0) * (uK - S);
    *u = S - c;
  }
  const double ratio = c / cK;
  *rho = rhoK * pow(ratio, 2.0 / (g - 1.0));
  *p = pK * pow(ratio, 2.0 * g / (g - 1.0));
}

/* one side adjoining vacuum (dir=-1: left state facing vacuum on its right) */
static void sample_vacuum_side(double g, double rhoK, double uK, double pK, int dir, double S, double* out) {
  const double cK = sqrt(g * pK / rhoK);
  if (dir < 0) { /* left state, vacuum to the right: left-facing fan */
    const double head = uK - cK, front = uK + 2.0 * cK / (g - 1.0);
    if (S <= head) {
      out[0] = rhoK; out[1] = uK; out[2] = pK;
    } else if (S >= front) {
      out[0] = 0.0; out[1] = front; out[2] = 0.0;
    } else {
      fan_state(g, rhoK, uK, pK, cK, -1, S, &out[0], &out[1], &out[2]);
    }
  } else { /* right state, vacuum to the left: right-facing fan */
    const double head = uK + cK, front = uK - 2.0 * cK / (g - 1.0);
    if (S >= head) {
      out[0] = rhoK; out[1] = uK; out[2] = pK;
    } else if (S <= front) {
      out[0] = 0.0; out[1] = front; out[2] = 0.0;
    } else {
      fan_state(g, rhoK, uK, pK, cK, +1, S, &out[0], &out[1], &out[2]);
    }
  }
}

int ora_riemann(double g, const double* WL, const double* WR, double tol, int maxit, double* out, int* niter) {
  const double rhoL = WL[0], uL = WL[1], pL = WL[2];
  const double rhoR = WR[0], uR = WR[1], pR = WR[2];
  const double S = 0.0;
  *niter = 0;
  /* vacuum on one or both sides */
  if (!(rhoL > 0.0) && !(rhoR > 0.0)) {
    out[0] = out[1] = out[2] = out[3] = out[4] = 0.0;
    out[5] = 0.0;
    return 1;
  }
  if (!(rhoL > 0.0)) {
    sample_vacuum_side(g, rhoR, uR, pR, +1, S, out);
    out[3] = 0.0;
    out[4] = uR - 2.0 * sqrt(g * pR / rhoR) / (g - 1.0);
    out[5] = 1.0;
    return 1;
  }
  if (!(rhoR > 0.0)) {
    sample_vacuum_side(g, rhoL, uL, pL, -1, S, out);
    out[3] = 0.0;
    out[4] = uL + 2.0 * sqrt(g * pL / rhoL) / (g - 1.0);
    out[5] = 0.0;
    return 1;
  }
  const double cL = sqrt(g * pL / rhoL), cR = sqrt(g * pR / rhoR);
  /* vacuum generated between two rarefactions */
  if (2.0 * (cL + cR) / (g - 1.0) <= uR - uL) {
    const double frontL = uL + 2.0 * cL / (g - 1.0);
    const double frontR = uR - 2.0 * cR / (g - 1.0);
    if (S <= frontL) {
      sample_vacuum_side(g, rhoL, uL, pL, -1, S, out);
      out[5] = 0.0;
    } else if (S >= frontR) {
      sample_vacuum_side(g, rhoR, uR, pR, +1, S, out);
      out[5] = 1.0;
    } else {
      out[0] = 0.0; out[1] = 0.5 * (frontL + frontR); out[2] = 0.0;
      out[5] = 0.0;
    }
    out[3] = 0.0;
    out[4] = 0.5 * (frontL + frontR);
    return 1;
  }
  /* initial guess: adaptive choice among the linearised (primitive-variable),
   * two-rarefaction and two-shock estimates, switch ratio 2 */
  const double du = uR - uL;
  double p0;
  {
    const double ppv0 = 0.5 * (pL + pR) - 0.125 * du * (rhoL + rhoR) * (cL + cR);
    const double ppv = ppv0 > 0.0 ? ppv0 : 0.0;
    const double pmin = pL < pR ? pL : pR, pmax = pL > pR ? pL : pR;
    if (pmax / pmin <= 2.0 && ppv >= pmin && ppv <= pmax) {
      p0 = ppv;
    } else if (ppv < pmin) {
      const double z = (g - 1.0) / (2.0 * g);
      const double num = cL + cR - 0.5 * (g - 1.0) * du;
      const double den = cL / pow(pL, z) + cR / pow(pR, z);
      p0 = pow(num / den, 1.0 / z);
    } else {
      const double AL = 2.0 / ((g + 1.0) * rhoL), BL = (g - 1.0) / (g + 1.0) * pL;
      const double AR = 2.0 / ((g + 1.0) * rhoR), BR = (g - 1.0) / (g + 1.0) * pR;
      const double gL = sqrt(AL / (ppv + BL)), gR = sqrt(AR / (ppv + BR));
      p0 = (gL * pL + gR * pR - du) / (gL + gR);
    }
    const double pfloor = 1e-10 * 0.5 * (pL + pR);
    if (!(p0 > pfloor)) p0 = pfloor;
  }
  /* Newton iteration on f(p) = 0; it also stops when f(p) vanishes to
   * rounding (|f| within 64 ulps of the size of its terms): p is then the root
   * in working precision.  Near vacuum f is a small difference of large terms
   * and the relative change of p cannot fall below tol. */
  double p = p0;
  int it = 0, conv = 0;
  while (it < maxit) {
    double dL, dR;
    const double fLp = pfun(p, rhoL, pL, cL, g, &dL), fRp = pfun(p, rhoR, pR, cR, g, &dR);
    const double f = fLp + fRp + du;
    if (fabs(f) <= 64.0 * DBL_EPSILON * (fabs(fLp) + fabs(fRp) + fabs(du))) {
      conv = 1;
      break;
    }
    double pn = p - f / (dL + dR);
    if (!(pn > 0.0)) pn = 1e-3 * p;
    it++;
    const double change = 2.0 * fabs(pn - p) / (pn + p);
    p = pn;
    if (change < tol) {
      conv = 1;
      break;
    }
  }
  *niter = it;
  double dL, dR;
  const double fL = pfun(p, rhoL, pL, cL, g, &dL), fR = pfun(p, rhoR, pR, cR, g, &dR);
  const double us = 0.5 * (uL + uR) + 0.5 * (fR - fL);
  out[3] = p;
  out[4] = us;
  /* sample at x/t = S */
  if (S <= us) { /* left of the contact */
    out[5] = 0.0;
    if (p > pL) { /* left shock */
      const double SL = uL - cL * sqrt((g + 1.0) / (2.0 * g) * p / pL + (g - 1.0) / (2.0 * g));
      if (S <= SL) {
        out[0] = rhoL; out[1] = uL; out[2] = pL;
      } else {
        const double r = p / pL, g6 = (g - 1.0) / (g + 1.0);
        out[0] = rhoL * (r + g6) / (g6 * r + 1.0); out[1] = us; out[2] = p;
      }
    } else { /* left rarefaction */
      const double head = uL - cL;
      const double cs = cL * pow(p / pL, (g - 1.0) / (2.0 * g));
      const double tail = us - cs;
      if (S <= head) {
        out[0] = rhoL; out[1] = uL; out[2] = pL;
      } else if (S > tail) {
        out[0] = rhoL * pow(p / pL, 1.0 / g); out[1] = us; out[2] = p;
      } else {
        fan_state(g, rhoL, uL, pL, cL, -1, S, &out[0], &out[1], &out[2]);
      }
    }
  } else { /* right of the contact */
    out[5] = 1.0;
    if (p > pR) { /* right shock */
      const double SR = uR + cR * sqrt((g + 1.0) / (2.0 * g) * p / pR + (g - 1.0) / (2.0 * g));
      if (S >= SR) {
        out[0] = rhoR; out[1] = uR; out[2] = pR;
      } else {
        const double r = p / pR, g6 = (g - 1.0) / (g + 1.0);
        out[0] = rhoR * (r + g6) / (g6 * r + 1.0); out[1] = us; out[2] = p;
      }
    } else { /* right rarefaction */
      const double head = uR + cR;
      const double cs = cR * pow(p / pR, (g - 1.0) / (2.0 * g));
      const double tail = us + cs;
      if (S >= head) {
        out[0] = rhoR; out[1] = uR; out[2] = pR;
      } else if (S < tail) {
        out[0] = rhoR * pow(p / pR, 1.0 / g); out[1] = us; out[2] = p;
      } else {
        fan_state(g, rhoR, uR, pR, cR, +1, S, &out[0], &out[1], &out[2]);
      }
    }
  }
  return conv ? 0 : -1;
}

/* batch form for tests: W* arrays [m][3], out [m][6], niter [m]; returns
 * the number of problems that did not converge */
long ora_riemann_batch(double g, long m, const double* WL, const double* WR, double tol, int maxit, double* out,
                       int32_t* niter) {
  long bad = 0;
  for (long q = 0; q < m; q++) {
    int it = 0;
    if (ora_riemann(g, WL + 3 * q, WR + 3 * q, tol, maxit, out + 6 * q, &it) < 0) bad++;
    niter[q] = it;
  }
  return bad;
}

/* ------------------------------------------------------ A5: face velocity
 * Sec. 3.3 (Fig. FigSketchVelFace): w = (w_L + w_R)/2 + w', with
 * w' = [(w_L - w_R) . (f - (r_R + r_L)/2)] / |r_R - r_L| * (r_R - r_L)/|r_R - r_L|.
 * wface: [nf][dim].  wmesh NULL means a static mesh. */
typedef struct {
  int dim;
  const int32_t* cells;
  const int8_t* shift;
  const double *gen, *cen, *box, *wmesh;
  double* wface;
} fv_args;

static void fv_face(const void* a, long k, int64_t* counters) {
  (void)counters;
  const fv_args* A = (const fv_args*)a;
  const int dim = A->dim;
  const int32_t* cells = A->cells;
  const int8_t* shift = A->shift;
  const double *gen = A->gen, *cen = A->cen, *box = A->box, *wmesh = A->wmesh;
  double* wface = A->wface;
  {
    const int L = cells[2 * k], R = cells[2 * k + 1];
    double rL[3], rR[3];
    face_positions(dim, k, gen, cells, shift, box, rL, rR);
    double sep = 0.0;
    for (int d = 0; d < dim; d++) sep += (rR[d] - rL[d]) * (rR[d] - rL[d]);
    sep = sqrt(sep);
    double proj = 0.0;
    for (int d = 0; d < dim; d++) {
      const double wL = wmesh ? wmesh[(long)L * dim + d] : 0.0;
      const double wR = wmesh ? wmesh[(long)R * dim + d] : 0.0;
      proj += (wL - wR) * (cen[k * dim + d] - 0.5 * (rR[d] + rL[d]));
    }
    for (int d = 0; d < dim; d++) {
      const double wL = wmesh ? wmesh[(long)L * dim + d] : 0.0;
      const double wR = wmesh ? wmesh[(long)R * dim + d] : 0.0;
      wface[k * dim + d] = 0.5 * (wR + wL) + proj / sep * (rR[d] - rL[d]) / sep;
    }
  }
}

void ora_face_velocities(int dim, long nf, const int32_t* cells, const int8_t* shift, const double* gen,
                         const double* cen, const double* box, const double* wmesh, double* wface) {
  const fv_args A = {dim, cells, shift, gen, cen, box, wmesh, wface};
  par_for(nf, fv_face, &A, NULL);
}

/* ------------------------------------------------- A6: MUSCL-Hancock flux
 * Sec. 3.3, eqs. (eqnrefframe) to (eqfinalflux), for every face:
 *  1. W'_K = W_K - (0, w, 0): the cell-centre state in the face frame;
 *  2. W''_K = W'_K + dW/dr|_K (f - s_K) + dW'/dt|_K dt/2, with the time
 *     derivative from dW/dt = -A(W) dW/dr evaluated at the cell-centre state
 *     W'_K in the face frame (component form:
 *       drho/dt = -(v'.grad rho + rho div v),
 *       dv/dt   = -(v'.grad) v - grad P / rho,
 *       dP/dt   = -(gamma P div v + v'.grad P));
 *     if either side's rho'' or P'' is not positive, both sides fall back to
 *     W' (first order) and the face is counted;
 *  3. rotate: normal velocity u = v''.n, transverse vector v'' - u n kept;
 *  4. Riemann problem along n, sampled at x/t = 0; transverse velocity taken
 *     from the side of the contact that x/t = 0 lies on (the left side when
 *     u* = 0);
 *  5. back to the lab frame v_lab = u_F n + v_t + w and the flux of the
 *     moving face, projected on n:
 *       F_m = rho_F u_F,  F_p = rho_F v_lab u_F + P_F n,
 *       F_E = (rho_F |v_lab|^2/2 + P_F/(gamma-1)) u_F + P_F v_lab . n.
 * F: [nf][dim+2] per unit area (not multiplied by A).
 * counters: [0] fallback faces, [1] vacuum faces, [2] Newton iterations,
 * [3] Newton failures.  Returns 0, or -1 if any Newton solve failed. */
typedef struct {
  int dim;
  const double *W, *grad, *gen, *s, *wface;
  const int32_t* cells;
  const int8_t* shift;
  const double *cen, *box;
  double gamma, dt, tol;
  int maxit;
  double* F;
  double* FS;  /* entropy flux per unit area (Sec. 3.5), or NULL */
  double* MF;  /* largest shock Mach number of the face's Riemann problem, or NULL */
  const double* Acell;  /* entropic function A = S/M per cell (with FS) */
  const double* gA;     /* its limited gradient [n][dim] (with FS) */
  const long* list;     /* if set: the loop index selects face list[index] */
  const double* hside;  /* if set: [nf][2] time of each side's prediction (else dt/2) */
} flux_args;

static void flux_face(const void* a, long k, int64_t* counters);

int ora_fluxes(int dim, long n, const double* W, const double* grad, const double* gen, const double* s,
               const double* wmesh, long nf, const int32_t* cells, const int8_t* shift, const double* area,
               const double* cen, const double* box, double gamma, double dt, double tol, int maxit, double* F,
               int64_t* counters) {
  (void)n;
  (void)area;
  double* wface = (double*)malloc(sizeof(double) * (size_t)(nf * dim + 1));
  ora_face_velocities(dim, nf, cells, shift, gen, cen, box, wmesh, wface);
  const flux_args A = {dim, W, grad, gen, s, wface, cells, shift, cen, box, gamma, dt, tol, maxit, F, NULL, NULL, NULL,
                       NULL, NULL, NULL};
  const int64_t fails_before = counters[3];
  par_for(nf, flux_face, &A, counters);
  free(wface);
  return counters[3] > fails_before ? -1 : 0;
}

static void flux_face(const void* a, long idx, int64_t* counters) {
  const flux_args* A = (const flux_args*)a;
  const long k = A->list ? A->list[idx] : idx;
  const int dim = A->dim;
  const double *W = A->W, *grad = A->grad, *gen = A->gen, *s = A->s, *wface = A->wface;
  const int32_t* cells = A->cells;
  const int8_t* shift = A->shift;
  const double *cen = A->cen, *box = A->box;
  const double gamma = A->gamma, dt = A->dt, tol = A->tol;
  const int maxit = A->maxit;
  double* F = A->F;
  const int nv = dim + 2;
  {
    const int cellK[2] = {cells[2 * k], cells[2 * k + 1]};
    double rL[3], rR[3];
    face_positions(dim, k, gen, cells, shift, box, rL, rR);
    double nrm[3], sep = 0.0;
    for (int d = 0; d < dim; d++) sep += (rR[d] - rL[d]) * (rR[d] - rL[d]);
    sep = sqrt(sep);
    for (int d = 0; d < dim; d++) nrm[d] = (rR[d] - rL[d]) / sep;
    const double* w = wface + k * dim;

    double Wp[2][NV_MAX], Wpp[2][NV_MAX];
    double App[2] = {0.0, 0.0}; /* entropic function at the face (Sec. 3.5) */
    for (int side = 0; side < 2; side++) {
      const long i = cellK[side];
      const double* Wi = W + i * nv;
      const double* gi = grad + i * nv * dim;
      /* face centroid relative to the centre of mass, in cell i's frame */
      double fs[3];
      for (int d = 0; d < dim; d++) {
        const double sh = (side == 1) ? shift[k * dim + d] * box[d] : 0.0;
        fs[d] = (cen[k * dim + d] - sh) - s[i * dim + d];
      }
      /* 1. boost into the face frame */
      Wp[side][0] = Wi[0];
      for (int d = 0; d < dim; d++) Wp[side][1 + d] = Wi[1 + d] - w[d];
      Wp[side][dim + 1] = Wi[dim + 1];
      /* 2a. spatial extrapolation to the face centroid */
      for (int v = 0; v < nv; v++) {
        double dv = 0.0;
        for (int d = 0; d < dim; d++) dv += gi[v * dim + d] * fs[d];
        Wpp[side][v] = Wp[side][v] + dv;
      }
      /* 2b. half-step time prediction with A(W') at the cell centre (over
       * hs = dt/2, or the side's own interval with individual steps) */
      const double hs = A->hside ? A->hside[2 * k + side] : 0.5 * dt;
      const double rho = Wp[side][0], P = Wp[side][dim + 1];
      const double* vp = &Wp[side][1];
      double divv = 0.0, vgrad_rho = 0.0, vgrad_P = 0.0;
      for (int d = 0; d < dim; d++) {
        divv += gi[(1 + d) * dim + d];
        vgrad_rho += vp[d] * gi[0 * dim + d];
        vgrad_P += vp[d] * gi[(dim + 1) * dim + d];
      }
      const double drho_dt = -(vgrad_rho + rho * divv);
      const double dP_dt = -(gamma * P * divv + vgrad_P);
      Wpp[side][0] += hs * drho_dt;
      Wpp[side][dim + 1] += hs * dP_dt;
      for (int a = 0; a < dim; a++) {
        double adv = 0.0;
        for (int d = 0; d < dim; d++) adv += vp[d] * gi[(1 + a) * dim + d];
        const double dva_dt = -adv - gi[(dim + 1) * dim + a] / rho;
        Wpp[side][1 + a] += hs * dva_dt;
      }
      if (A->FS) {
        /* A reconstructed like the other primitives; it is advected,
         * dA/dt = -v'.grad A */
        const double* ga = A->gA + i * dim;
        double dA = 0.0, vgrad_A = 0.0;
        for (int d = 0; d < dim; d++) {
          dA += ga[d] * fs[d];
          vgrad_A += vp[d] * ga[d];
        }
        App[side] = A->Acell[i] + dA + hs * (-vgrad_A);
        if (!(App[side] > 0.0)) App[side] = A->Acell[i];
      }
    }
    if (!(Wpp[0][0] > 0.0) || !(Wpp[0][dim + 1] > 0.0) || !(Wpp[1][0] > 0.0) || !(Wpp[1][dim + 1] > 0.0)) {
      for (int side = 0; side < 2; side++)
        for (int v = 0; v < nv; v++) Wpp[side][v] = Wp[side][v];
      if (A->FS) {
        App[0] = A->Acell[cellK[0]];
        App[1] = A->Acell[cellK[1]];
      }
      counters[0]++;
    }
    /* 3. rotate: normal component and transverse vector */
    double un[2], vt[2][3];
    for (int side = 0; side < 2; side++) {
      double u = 0.0;
      for (int d = 0; d < dim; d++) u += Wpp[side][1 + d] * nrm[d];
      un[side] = u;
      for (int d = 0; d < dim; d++) vt[side][d] = Wpp[side][1 + d] - u * nrm[d];
    }
    /* 4. Riemann problem */
    const double WLr[3] = {Wpp[0][0], un[0], Wpp[0][dim + 1]};
    const double WRr[3] = {Wpp[1][0], un[1], Wpp[1][dim + 1]};
    double out[6];
    int it = 0;
    const int st = ora_riemann(gamma, WLr, WRr, tol, maxit, out, &it);
    counters[2] += it;
    if (st < 0) counters[3]++;
    if (st == 1) counters[1]++;
    const double rhoF = out[0], uF = out[1], PF = out[2];
    const int up = (out[5] > 0.5) ? 1 : 0;
    /* 5. back to the lab frame and the flux of the moving face */
    double vlab[3], v2 = 0.0, vn = 0.0;
    for (int d = 0; d < dim; d++) {
      vlab[d] = uF * nrm[d] + vt[up][d] + w[d];
      v2 += vlab[d] * vlab[d];
      vn += vlab[d] * nrm[d];
    }
    double* Fk = F + k * nv;
    Fk[0] = rhoF * uF;
    for (int d = 0; d < dim; d++) Fk[1 + d] = rhoF * vlab[d] * uF + PF * nrm[d];
    Fk[dim + 1] = (0.5 * rhoF * v2 + PF / (gamma - 1.0)) * uF + PF * vn;
    if (A->FS) {
      /* Sec. 3.5: entropy flux rho_F u_F A_U with A_U the reconstructed
       * entropic function of the upwind side; shock Mach numbers of the
       * waves with p* above the pressure ahead of them */
      A->FS[k] = rhoF * uF * ((uF > 0.0) ? App[0] : App[1]);
      double mach = 1.0;
      if (st == 0) {
        const double ps = out[3];
        for (int side = 0; side < 2; side++) {
          const double pK = Wpp[side][dim + 1];
          if (ps > pK) {
            const double m = sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (ps / pK - 1.0));
            if (m > mach) mach = m;
          }
        }
      }
      A->MF[k] = mach;
    }
  }
}

/* the same fluxes, plus the entropy flux and the face's shock Mach number;
 * Acell: A = S/M per cell, gA: its limited gradient [n][dim] */
int ora_fluxes_entropy(int dim, long n, const double* W, const double* grad, const double* gen, const double* s,
                       const double* wmesh, long nf, const int32_t* cells, const int8_t* shift, const double* area,
                       const double* cen, const double* box, double gamma, double dt, double tol, int maxit,
                       const double* Acell, const double* gA, double* F, double* FS, double* MF,
                       int64_t* counters) {
  (void)n;
  (void)area;
  double* wface = (double*)malloc(sizeof(double) * (size_t)(nf * dim + 1));
  ora_face_velocities(dim, nf, cells, shift, gen, cen, box, wmesh, wface);
  const flux_args A = {dim, W, grad, gen, s, wface, cells, shift, cen, box, gamma, dt, tol, maxit, F, FS, MF,
                       Acell, gA, NULL, NULL};
  const int64_t fails_before = counters[3];
  par_for(nf, flux_face, &A, counters);
  free(wface);
  return counters[3] > fails_before ? -1 : 0;
}

/* ------------------------------------------------- A8: conservative update
 * Eq. (eqnupdate): Q_i^{n+1} = Q_i^n - dt sum_j A_ij F_ij, where the flux
 * F_ij leaves cell i through face (i,j); with the face normal pointing from
 * L to R that is +F for the left cell and -F for the right cell. */
typedef struct {
  int dim;
  const double *Q, *area, *F;
  double dt;
  double* Qnew;
  const incidence* I;
} upd_args;

static void upd_cell(const void* a, long i, int64_t* counters);

void ora_update(int dim, long n, const double* Q, long nf, const int32_t* cells, const double* area,
                const double* F, double dt, double* Qnew) {
  incidence I = build_incidence(n, nf, cells);
  const upd_args A = {dim, Q, area, F, dt, Qnew, &I};
  par_for(n, upd_cell, &A, NULL);
  free_incidence(&I);
}

static void upd_cell(const void* a, long i, int64_t* counters) {
  (void)counters;
  const upd_args* A = (const upd_args*)a;
  const int dim = A->dim;
  const double *Q = A->Q, *area = A->area, *F = A->F;
  const double dt = A->dt;
  double* Qnew = A->Qnew;
  const incidence I = *A->I;
  const int nv = dim + 2;
  {
    double sum[NV_MAX] = {0, 0, 0, 0, 0};
    for (long q = I.off[i]; q < I.off[i + 1]; q++) {
      const long k = I.face[q];
      const double sgn = (I.side[q] == 0) ? 1.0 : -1.0;
      for (int v = 0; v < nv; v++) sum[v] += sgn * area[k] * F[k * nv + v];
    }
    for (int v = 0; v < nv; v++) Qnew[i * nv + v] = Q[i * nv + v] - dt * sum[v];
  }
}

/* ------------------------------- Sec. 3.5: entropy and the shock switch
 * S_i = M_i A_i with the entropic function A = P / rho^gamma is advected as
 * a further conserved quantity with the face fluxes rho_F u_F A_U.  At the
 * end of the step each cell either keeps the advected entropy (when the
 * largest shock Mach number among the Riemann problems of its faces is below
 * mach_thresh: the flow around it is smooth; or, with alpha_s > 0, when the
 * new thermal energy is below alpha_s times the largest kinetic energy around
 * it: the flow is cold) and sets its thermal energy from it,
 * P = (S/M) rho^gamma, E = M |v|^2/2 + P V/(gamma-1); or it keeps
 * the conservative energy update and re-initialises S = M P / rho^gamma.
 * Q, Qnew: [n][dim+2]; S, Snew: [n]; kept[i] = 1 where the entropy was kept. */
void ora_entropy_init(int dim, long n, const double* Q, const double* V, double gamma, double* S) {
  const int nv = dim + 2;
  for (long i = 0; i < n; i++) {
    const double m = Q[i * nv];
    const double rho = m / V[i];
    double v2 = 0.0;
    for (int d = 0; d < dim; d++) {
      const double v = Q[i * nv + 1 + d] / m;
      v2 += v * v;
    }
    const double P = (gamma - 1.0) * (Q[i * nv + dim + 1] / V[i] - 0.5 * rho * v2);
    S[i] = m * P / pow(rho, gamma);
  }
}

typedef struct {
  int dim;
  const double *Q, *S, *V, *area, *F, *FS, *MF, *wmesh;
  const int32_t* cells;
  double dt, gamma, mach_thresh, alpha_s;
  double *Qnew, *Snew;
  int32_t* kept;
  const incidence* I;
} ent_args;

static void ent_cell(const void* a, long i, int64_t* counters) {
  const ent_args* A = (const ent_args*)a;
  const int dim = A->dim;
  const int nv = dim + 2;
  const incidence I = *A->I;
  double sum[NV_MAX] = {0, 0, 0, 0, 0}, sumS = 0.0, mach = 1.0;
  for (long q = I.off[i]; q < I.off[i + 1]; q++) {
    const long k = I.face[q];
    const double sgn = (I.side[q] == 0) ? 1.0 : -1.0;
    for (int v = 0; v < nv; v++) sum[v] += sgn * A->area[k] * A->F[k * nv + v];
    sumS += sgn * A->area[k] * A->FS[k];
    if (A->MF[k] > mach) mach = A->MF[k];
  }
  double* Qn = A->Qnew + i * nv;
  for (int v = 0; v < nv; v++) Qn[v] = A->Q[i * nv + v] - A->dt * sum[v];
  const double Sadv = A->S[i] - A->dt * sumS;
  const double m = Qn[0];
  const double V = A->V[i];
  const double rho = m / V;
  double p2 = 0.0;
  for (int d = 0; d < dim; d++) p2 += Qn[1 + d] * Qn[1 + d];
  /* cold-flow criterion, eq. (eqnScrit1): the new thermal energy against the
   * largest kinetic energy of the cell and its neighbours (start-of-step
   * states), measured relative to the cell's own mesh velocity */
  int cold = 0;
  if (A->alpha_s > 0.0) {
    double ekmax = 0.0;
    for (long q = I.off[i] - 1; q < I.off[i + 1]; q++) {
      const long j = (q < I.off[i]) ? i : (long)A->cells[2 * I.face[q] + (1 - I.side[q])];
      const double mj = A->Q[j * nv];
      double dv2 = 0.0;
      for (int d = 0; d < dim; d++) {
        const double dv = A->Q[j * nv + 1 + d] / mj - (A->wmesh ? A->wmesh[i * dim + d] : 0.0);
        dv2 += dv * dv;
      }
      const double ek = 0.5 * mj * dv2;
      if (ek > ekmax) ekmax = ek;
    }
    const double eth = Qn[dim + 1] - 0.5 * p2 / m;
    cold = eth < A->alpha_s * ekmax;
  }
  if (mach < A->mach_thresh || cold) {
    const double P = (Sadv / m) * pow(rho, A->gamma);
    Qn[dim + 1] = 0.5 * p2 / m + P * V / (A->gamma - 1.0);
    A->Snew[i] = Sadv;
    A->kept[i] = 1;
    counters[0]++;
  } else {
    const double P = (A->gamma - 1.0) * (Qn[dim + 1] / V - 0.5 * p2 / (m * V));
    A->Snew[i] = m * P / pow(rho, A->gamma);
    A->kept[i] = 0;
  }
}

/* one whole step with the entropy switch; as ora_step, plus S in/out, the
 * shock-Mach threshold, the cold-flow parameter alpha_s (0: off), and
 * counters[4] = cells that kept their entropy */
int ora_step_entropy(int dim, long n, const double* gen, long nf, const int32_t* cells, const int8_t* shift,
                     const double* area, const double* cen, const double* box, const double* V, const double* s,
                     const double* Q, const double* S, double gamma, int mode, const double* wmesh_in, double dt,
                     double cfl, int limit, double tol, int maxit, double mach_thresh, double alpha_s, double* Qnew,
                     double* Snew, int32_t* kept, double* dt_used, int64_t* counters) {
  const int nv = dim + 2;
  double* W = (double*)malloc(sizeof(double) * (size_t)(n * nv));
  double* grad = (double*)malloc(sizeof(double) * (size_t)(n * nv * dim));
  double* wm = (double*)malloc(sizeof(double) * (size_t)(n * dim));
  double* F = (double*)malloc(sizeof(double) * (size_t)(nf * nv + 1));
  double* FS = (double*)malloc(sizeof(double) * (size_t)(nf + 1));
  double* MF = (double*)malloc(sizeof(double) * (size_t)(nf + 1));
  double* Wx = (double*)malloc(sizeof(double) * (size_t)(n * (nv + 1)));
  double* gx = (double*)malloc(sizeof(double) * (size_t)(n * (nv + 1) * dim));
  double* Ac = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  double* gA = (double*)malloc(sizeof(double) * (size_t)(n * dim + 1));
  ora_primitives(dim, n, Q, V, gamma, W);
  /* the primitives and the entropic function A = S/M, gradients and limiter
   * per variable (the first nv exactly as in ora_gradients) */
  for (long i = 0; i < n; i++) {
    for (int v = 0; v < nv; v++) Wx[i * (nv + 1) + v] = W[i * nv + v];
    Ac[i] = S[i] / Q[i * nv];
    Wx[i * (nv + 1) + nv] = Ac[i];
  }
  gradients_nvar(dim, n, nv + 1, Wx, gen, V, s, nf, cells, shift, area, cen, box, limit, gx);
  for (long i = 0; i < n; i++) {
    for (int v = 0; v < nv; v++)
      for (int d = 0; d < dim; d++) grad[(i * nv + v) * dim + d] = gx[(i * (nv + 1) + v) * dim + d];
    for (int d = 0; d < dim; d++) gA[i * dim + d] = gx[(i * (nv + 1) + nv) * dim + d];
  }
  for (long i = 0; i < n; i++)
    for (int d = 0; d < dim; d++)
      wm[i * dim + d] = (mode == 0) ? 0.0 : (mode == 1) ? W[i * nv + 1 + d] : wmesh_in[i * dim + d];
  if (!(dt > 0.0)) dt = ora_timestep(dim, n, W, V, wm, gamma, cfl, NULL);
  *dt_used = dt;
  for (int c = 0; c < 5; c++) counters[c] = 0;
  const int rc = ora_fluxes_entropy(dim, n, W, grad, gen, s, wm, nf, cells, shift, area, cen, box, gamma, dt, tol,
                                    maxit, Ac, gA, F, FS, MF, counters);
  free(Wx);
  free(gx);
  free(Ac);
  free(gA);
  incidence I = build_incidence(n, nf, cells);
  const ent_args A = {dim, Q, S, V, area, F, FS, MF, wm, cells, dt, gamma, mach_thresh, alpha_s, Qnew, Snew, kept,
                      &I};
  int64_t c5[4] = {0, 0, 0, 0};
  par_for(n, ent_cell, &A, c5);
  counters[4] = c5[0];
  free_incidence(&I);
  free(W);
  free(grad);
  free(wm);
  free(F);
  free(FS);
  free(MF);
  return rc;
}

/* ------------------------------------------------ A9: conservation sums */
void ora_totals(int dim, long n, const double* Q, double* tot) {
  const int nv = dim + 2;
  for (int v = 0; v < nv; v++) tot[v] = 0.0;
  for (long i = 0; i < n; i++)
    for (int v = 0; v < nv; v++) tot[v] += Q[i * nv + v];
}

/* --------------------------------- Sec. 4.1: mesh-regularity correction
 * Eq. (EqnShapeCorrVel): a generator further than a fraction eta of its
 * cell's radius R_i = (3 V_i / 4 pi)^(1/3) (2D: (V_i / pi)^(1/2)) from the
 * centre of mass s_i is given an extra velocity towards it,
 *   w_i' = w_i + chi c_i (s_i - r_i)/d_i * ramp,  d_i = |s_i - r_i|,
 *   ramp = 0 for d_i < 0.9 eta R_i, (d_i - 0.9 eta R_i)/(0.2 eta R_i) up to
 *   1.1 eta R_i, 1 beyond; c_i = sqrt(gamma P_i / rho_i).
 * s: [n][dim] centres of mass in the cell's own frame (as ora_geometry
 * returns them); w, wout: [n][dim]. */
void ora_shape_correction(int dim, long n, const double* gen, const double* s, const double* V, const double* W,
                          const double* w, double gamma, double eta, double chi, double* wout) {
  const int nv = dim + 2;
  for (long i = 0; i < n; i++) {
    double d2 = 0.0, ds[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < dim; k++) {
      ds[k] = s[i * dim + k] - gen[i * dim + k];
      d2 += ds[k] * ds[k];
    }
    const double d = sqrt(d2);
    const double R = (dim == 3) ? cbrt(3.0 * V[i] / (4.0 * M_PI)) : sqrt(V[i] / M_PI);
    double ramp = 0.0;
    if (d >= 1.1 * eta * R)
      ramp = 1.0;
    else if (d >= 0.9 * eta * R)
      ramp = (d - 0.9 * eta * R) / (0.2 * eta * R);
    const double c = sqrt(gamma * W[i * nv + dim + 1] / W[i * nv]);
    for (int k = 0; k < dim; k++) wout[i * dim + k] = w[i * dim + k] + ((ramp > 0.0) ? chi * c * ds[k] / d * ramp : 0.0);
  }
}

/* ---------------------------------------------------- A10: generator drift
 * Sec. 3, step 8: r_i <- r_i + w_i dt, wrapped back into the box. */
void ora_drift(int dim, long n, double* gen, const double* wmesh, const double* box, double dt) {
  for (long i = 0; i < n; i++)
    for (int d = 0; d < dim; d++) {
      double x = gen[i * dim + d] + wmesh[i * dim + d] * dt;
      x = fmod(x, box[d]);
      if (x < 0.0) x += box[d];
      if (x >= box[d]) x -= box[d];
      gen[i * dim + d] = x;
    }
}

/* ------------------------------------------------------- one whole step
 * Sec. 3, steps 2-7 on a given tessellation: primitives, gradients and
 * limiter, mesh velocities (mode 0 static, 1 w = v, 2 the given wmesh),
 * the time step (dt <= 0 means dt = CFL condition with coefficient cfl),
 * fluxes and the conservative update.  V, s are taken from ora_geometry.
 * Outputs Qnew; dt_used; counters as in ora_fluxes. */
int ora_step(int dim, long n, const double* gen, long nf, const int32_t* cells, const int8_t* shift,
             const double* area, const double* cen, const double* box, const double* V, const double* s,
             const double* Q, double gamma, int mode, const double* wmesh_in, double dt, double cfl, int limit,
             double tol, int maxit, double* Qnew, double* dt_used, int64_t* counters) {
  const int nv = dim + 2;
  double* W = (double*)malloc(sizeof(double) * (size_t)(n * nv));
  double* grad = (double*)malloc(sizeof(double) * (size_t)(n * nv * dim));
  double* wm = (double*)malloc(sizeof(double) * (size_t)(n * dim));
  double* F = (double*)malloc(sizeof(double) * (size_t)(nf * nv + 1));
  ora_primitives(dim, n, Q, V, gamma, W);
  ora_gradients(dim, n, W, gen, V, s, nf, cells, shift, area, cen, box, limit, grad);
  for (long i = 0; i < n; i++)
    for (int d = 0; d < dim; d++)
      wm[i * dim + d] = (mode == 0) ? 0.0 : (mode == 1) ? W[i * nv + 1 + d] : wmesh_in[i * dim + d];
  if (!(dt > 0.0)) dt = ora_timestep(dim, n, W, V, wm, gamma, cfl, NULL);
  *dt_used = dt;
  for (int c = 0; c < 4; c++) counters[c] = 0;
  const int rc = ora_fluxes(dim, n, W, grad, gen, s, wm, nf, cells, shift, area, cen, box, gamma, dt, tol, maxit,
                            F, counters);
  ora_update(dim, n, Q, nf, cells, area, F, dt, Qnew);
  free(W);
  free(grad);
  free(wm);
  free(F);
  return rc;
}

/* ------------------------- Sec. 7.1: the signal-speed time step criterion
 * Eq. (EqnTiStepIndividual):
 *   dt_i = C min(tau_i, R_i / (c_i + |v_i|)),
 *   tau_i = min_{j != i} r_ij / (c_i + c_j - v_ij . r_ij / r_ij),
 * on a static mesh (w = 0), with r_ij = r_i - r_j to the nearest periodic
 * image of j (a component of exactly half the box keeps its sign),
 * v_ij = v_i - v_j, and the pairs whose signal speed is not positive (they
 * recede faster than sound can cross) left out.  The minimum is taken over
 * all cells by brute force.  signal = 0 drops tau (eq. EqnTiStep alone).
 * dt: [n]. */
typedef struct {
  int dim;
  long n;
  const double *gen, *box, *W, *V, *c;
  double cfl;
  int signal;
  double* dt;
} sig_args;

static void sig_cell(const void* a, long i, int64_t* counters) {
  (void)counters;
  const sig_args* A = (const sig_args*)a;
  const int dim = A->dim, nv = dim + 2;
  const double* W = A->W;
  const double R = (dim == 3) ? cbrt(3.0 * A->V[i] / (4.0 * M_PI)) : sqrt(A->V[i] / M_PI);
  double v2 = 0.0;
  for (int d = 0; d < dim; d++) v2 += W[i * nv + 1 + d] * W[i * nv + 1 + d];
  const double tloc = R / (A->c[i] + sqrt(v2));
  double tau = INFINITY;
  if (A->signal) {
    for (long j = 0; j < A->n; j++) {
      if (j == i) continue;
      double dx[3], r2 = 0.0, vr = 0.0;
      for (int d = 0; d < dim; d++) {
        const double L = A->box[d];
        dx[d] = A->gen[i * dim + d] - A->gen[j * dim + d];
        if (dx[d] > 0.5 * L)
          dx[d] -= L;
        else if (dx[d] < -0.5 * L)
          dx[d] += L;
        r2 += dx[d] * dx[d];
      }
      for (int d = 0; d < dim; d++) vr += (W[i * nv + 1 + d] - W[j * nv + 1 + d]) * dx[d];
      const double r = sqrt(r2);
      const double sig = A->c[i] + A->c[j] - vr / r;
      if (sig > 0.0) {
        const double t = r / sig;
        if (t < tau) tau = t;
      }
    }
  }
  A->dt[i] = A->cfl * (tau < tloc ? tau : tloc);
}

void ora_signal_timestep(int dim, long n, const double* gen, const double* box, const double* W, const double* V,
                         double gamma, double cfl, int signal, double* dt) {
  const int nv = dim + 2;
  double* c = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  for (long i = 0; i < n; i++) c[i] = sqrt(gamma * W[i * nv + dim + 1] / W[i * nv]);
  const sig_args A = {dim, n, gen, box, W, V, c, cfl, signal, dt};
  par_for(n, sig_cell, &A, NULL);
  free(c);
}

/* --------------------------------- Sec. 7.2: individual time steps
 * One cycle of length dt_max on a static mesh.  Cell time steps are
 * dt_max / 2^b (bin b = 0..max_depth): the largest such step not above the
 * cell's criterion dt_i.  Time runs in integer ticks of dt_max / 2^max_depth;
 * a cell is active at tick t when its step divides t, i.e. a step of its
 * starts there; every cell is active at t = 0.  At each tick with active
 * cells:
 *  1. active cells take their primitives from their conserved quantities,
 *     then their limited gradients (neighbours that are not active enter
 *     with the primitives of their own last activation) and their criterion
 *     (signal-speed form if `signal`, with the other cells' current
 *     primitives), and pick a bin: a smaller step is always allowed; a larger
 *     one is at most twice the current step, and only where that step also
 *     starts at this tick;
 *  2. every face with an active cell is integrated over the smaller step of
 *     its two cells, from this tick; each side is predicted to the middle of
 *     that interval from the primitives and gradients of its own last
 *     activation (the half-step prediction over the time since then);
 *  3. both cells of such a face exchange dt_f A F (pairwise, conservative);
 *  4. time moves to the next tick at which a step starts, the next multiple
 *     of the smallest step in use.
 * On return every cell has completed its last step at dt_max.
 * bins: [n] the bins in use at the end.  counters: [0..3] as in ora_fluxes,
 * [4] sub-steps, [5] face flux evaluations, [6] cell activations.
 * Returns 0, -1 if a Newton solve failed, -2 if a cell's criterion is below
 * dt_max / 2^max_depth (1 <= max_depth <= 40). */
static int64_t step_ticks(int max_depth, int b) { return (int64_t)1 << (max_depth - b); }

int ora_advance_individual(int dim, long n, const double* gen, long nf, const int32_t* cells,
                           const int8_t* shift, const double* area, const double* cen, const double* box,
                           const double* V, const double* s, const double* Q, double gamma, double cfl,
                           double dt_max, int max_depth, int signal, int limit, double tol, int maxit,
                           double* Qnew, int32_t* bins, int64_t* counters) {
  if (max_depth < 1 || max_depth > 40 || !(dt_max > 0.0)) return -2;
  const int nv = dim + 2;
  const int64_t T = (int64_t)1 << max_depth;
  const double dtick = dt_max / (double)T;
  double* W = (double*)calloc((size_t)(n * nv + 1), sizeof(double));
  double* Wt = (double*)malloc(sizeof(double) * (size_t)(n * nv + 1));
  double* grad = (double*)calloc((size_t)(n * nv * dim + 1), sizeof(double));
  double* gt = (double*)malloc(sizeof(double) * (size_t)(n * nv * dim + 1));
  double* dtc = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  double* F = (double*)malloc(sizeof(double) * (size_t)(nf * nv + 1));
  double* hside = (double*)malloc(sizeof(double) * (size_t)(2 * nf + 1));
  double* dtf = (double*)malloc(sizeof(double) * (size_t)(nf + 1));
  double* wzero = (double*)calloc((size_t)(n * dim + 1), sizeof(double));
  long* list = (long*)malloc(sizeof(long) * (size_t)(nf + 1));
  char* act = (char*)malloc((size_t)(n + 1));
  char* fact = (char*)malloc((size_t)(nf + 1));
  double* wface = (double*)malloc(sizeof(double) * (size_t)(nf * dim + 1));
  incidence I = build_incidence(n, nf, cells);
  for (int c = 0; c < 7; c++) counters[c] = 0;
  memcpy(Qnew, Q, sizeof(double) * (size_t)(n * nv));
  for (long i = 0; i < n; i++) bins[i] = 0;
  ora_face_velocities(dim, nf, cells, shift, gen, cen, box, wzero, wface); /* static mesh: all zero */
  int rc = 0;
  int64_t tick = 0;
  while (tick < T && rc == 0) {
    /* 1. activation */
    for (long i = 0; i < n; i++) act[i] = (tick % step_ticks(max_depth, bins[i]) == 0);
    ora_primitives(dim, n, Qnew, V, gamma, Wt);
    for (long i = 0; i < n; i++)
      if (act[i]) memcpy(W + i * nv, Wt + i * nv, sizeof(double) * (size_t)nv);
    ora_gradients(dim, n, W, gen, V, s, nf, cells, shift, area, cen, box, limit, gt);
    for (long i = 0; i < n; i++)
      if (act[i]) memcpy(grad + i * nv * dim, gt + i * nv * dim, sizeof(double) * (size_t)(nv * dim));
    ora_signal_timestep(dim, n, gen, box, W, V, gamma, cfl, signal, dtc);
    for (long i = 0; i < n && rc == 0; i++) {
      if (!act[i]) continue;
      counters[6]++;
      int b = 0;
      double st = dt_max;
      while (st > dtc[i]) {
        st *= 0.5;
        b++;
      }
      if (b > max_depth) {
        rc = -2;
        break;
      }
      if (tick == 0 || b >= bins[i])
        bins[i] = b;
      else if (tick % step_ticks(max_depth, bins[i] - 1) == 0)
        bins[i] = bins[i] - 1; /* twice the step, where that step starts now */
    }
    if (rc != 0) break;
    /* 2. the faces of this tick */
    long na = 0;
    for (long k = 0; k < nf; k++) {
      const long L = cells[2 * k], R = cells[2 * k + 1];
      fact[k] = act[L] || act[R];
      if (!fact[k]) continue;
      const int64_t sL = step_ticks(max_depth, bins[L]), sR = step_ticks(max_depth, bins[R]);
      const int64_t sf = sL < sR ? sL : sR;
      dtf[k] = (double)sf * dtick;
      /* middle of [tick, tick + sf] minus each side's last activation, in
       * half ticks (integers, exact) */
      const int64_t startL = tick - tick % sL, startR = tick - tick % sR;
      hside[2 * k] = (double)(2 * tick + sf - 2 * startL) * (0.5 * dtick);
      hside[2 * k + 1] = (double)(2 * tick + sf - 2 * startR) * (0.5 * dtick);
      list[na++] = k;
    }
    const flux_args A = {dim, W, grad, gen, s, wface, cells, shift, cen, box, gamma, 0.0, tol, maxit, F,
                         NULL, NULL, NULL, NULL, list, hside};
    const int64_t fails_before = counters[3];
    par_for(na, flux_face, &A, counters);
    if (counters[3] > fails_before) rc = -1;
    /* 3. pairwise exchange over the active faces */
    for (long i = 0; i < n; i++) {
      double sum[NV_MAX] = {0, 0, 0, 0, 0, 0};
      int touched = 0;
      for (long q = I.off[i]; q < I.off[i + 1]; q++) {
        const long k = I.face[q];
        if (!fact[k]) continue;
        touched = 1;
        const double sgn = (I.side[q] == 0) ? 1.0 : -1.0;
        for (int v = 0; v < nv; v++) sum[v] += sgn * dtf[k] * area[k] * F[k * nv + v];
      }
      if (touched)
        for (int v = 0; v < nv; v++) Qnew[i * nv + v] -= sum[v];
    }
    counters[4]++;
    counters[5] += na;
    /* 4. the next tick */
    int64_t smin = T;
    for (long i = 0; i < n; i++) {
      const int64_t si = step_ticks(max_depth, bins[i]);
      if (si < smin) smin = si;
    }
    tick = (tick / smin + 1) * smin;
  }
  free_incidence(&I);
  free(W);
  free(Wt);
  free(grad);
  free(gt);
  free(dtc);
  free(F);
  free(hside);
  free(dtf);
  free(wzero);
  free(list);
  free(act);
  free(fact);
  free(wface);
  return rc;
}
