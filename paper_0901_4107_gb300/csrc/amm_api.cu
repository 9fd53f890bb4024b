// C ABI of libamm (declared in include/amm.h): context creation and
// validation, the per-step call sequence, CUDA-graph capture of a whole step,
// and the getters.  Host code only; kernels live in geometry.cu and
// hydro_f{32,64}.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "amm_internal.cuh"

using amm::R4;
using amm::Tile;

namespace {

int fail(amm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(amm_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, AMM_ERR_CUDA, m);
}

#define CU(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

void free_ctx(amm_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->ind_exec) cudaGraphExecDestroy(c->ind_exec);
  if (c->ind_graph) cudaGraphDestroy(c->ind_graph);
  amm::vor::work_free((amm::vor::TessWork*)c->tess_ws);
  for (cudaEvent_t ev : c->prof_ev)
    if (ev) cudaEventDestroy(ev);
  void* ptrs[] = {c->gen,   c->box,     c->Q,       c->lr,       c->csr_off, c->csr,     c->ctiles,
                  c->ftiles, c->box_first_ctile, c->fgeo, c->igAB, c->cgeo64, c->cw,     c->grad, c->cwp, c->Apw,
                  c->wmesh, c->cgeo, c->crad, c->flux,    c->fluxE,   c->cour_bits, c->fmax_bits, c->wcorr, c->S, c->Aw, c->gradA, c->fluxS, c->machf, c->ekmax, c->kept, c->cell_perm, c->face_perm, c->barrier, c->box_status, c->dt_box, c->dt_used, c->partial,
                  c->totals, c->stats,  c->closure, c->mlp,      c->defer_list, c->defer_count, c->scratch, c->counter,
                  c->ind_bin, c->ind_act, c->ind_list, c->ind_flist, c->ind_count, c->ind_fstamp, c->ind_cstamp,
                  c->ind_fdt, c->ind_hist, c->ind_slot_cell, c->ind_cell_slot, c->ind_leaf_off, c->ind_level_off,
                  c->ind_rec, c->ind_rec32, c->ind_node, c->ind_loop, c->geo_ws};
  for (void* p : ptrs)
    if (p) cudaFree(p);

  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  delete c;
}

template <typename F64, typename F32>
cudaError_t dispatch(amm_ctx* c, F64 f64, F32 f32) {
  return c->is_fp64() ? f64() : f32();
}

cudaError_t ensure_scratch(amm_ctx* c, size_t doubles) {
  if (c->scratch_size >= doubles) return cudaSuccess;
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_size = 0;
  cudaError_t e = cudaMalloc((void**)&c->scratch, sizeof(double) * doubles);
  if (e == cudaSuccess) c->scratch_size = doubles;
  return e;
}

cudaError_t mark(amm_ctx* c, int k) {
  if (!c->profiling) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(c->prof_ev[k], c->stream, cudaEventRecordExternal)
                                             : cudaEventRecord(c->prof_ev[k], c->stream);
}

// the Courant minimum and the gradients of a step; cfl > 0: its step is cfl
// times the Courant minimum, cfl == 0: dt_box (the static mesh's predicted
// records are taken over half of it)
cudaError_t run_gradients(amm_ctx* c, double cfl) {
  cudaError_t e = mark(c, 0);
  if (e != cudaSuccess) return e;
  e = dispatch(c, [&] { return amm::launch_gradients<double>(c, cfl); },
               [&] { return amm::launch_gradients<float>(c, cfl); });
  if (e != cudaSuccess) return e;
  return mark(c, 1);
}

// the step after the gradients: flux, update, totals; cfl > 0 takes the
// time step from the Courant minimum on the device, cfl == 0 from dt_box
cudaError_t run_step_tail(amm_ctx* c, double cfl) {
  cudaError_t e = dispatch(c, [&] { return amm::launch_flux<double>(c, cfl); },
                           [&] { return amm::launch_flux<float>(c, cfl); });
  if (e != cudaSuccess) return e;
  if ((e = mark(c, 2)) != cudaSuccess) return e;
  e = dispatch(c, [&] { return amm::launch_update<double>(c, cfl); }, [&] { return amm::launch_update<float>(c, cfl); });
  if (e != cudaSuccess) return e;
  if ((e = mark(c, 3)) != cudaSuccess) return e;
  e = dispatch(c, [&] { return amm::launch_finish<double>(c, cfl); }, [&] { return amm::launch_finish<float>(c, cfl); });
  if (e != cudaSuccess) return e;
  return mark(c, 4);
}

int check_status(amm_ctx* c) {
  amm::DeviceStats s;
  cudaError_t e = cudaMemcpy(&s, c->stats, sizeof(s), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read status");
  if (s.status & amm::ST_TIMEOUT) return fail(c, AMM_ERR_TIMEOUT, "a bounded device wait timed out");
  if (s.status & amm::ST_DEPTH)
    return fail(c, AMM_ERR_NUMERIC, "a cell's time-step criterion fell below dt_max / 2^max_depth");
  if (s.status & amm::ST_SUBSTEPS)
    return fail(c, AMM_ERR_NUMERIC, "a cycle of individual time steps exceeded 2^20 sub-steps");
  if (s.status & (amm::ST_NEWTON_CAP | amm::ST_NONPOS)) {
    char buf[256];
    snprintf(buf, sizeof buf, "numeric failure: %llu Newton solves hit the cap, %llu cells non-positive",
             (unsigned long long)s.newton_fail, (unsigned long long)s.nonpos);
    return fail(c, AMM_ERR_NUMERIC, buf);
  }
  return AMM_OK;
}

bool finite_all(const double* a, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

extern "C" {

void amm_default_options(amm_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = AMM_FP64;
  o->mesh_motion = AMM_LAGRANGIAN;
  o->limiter = 1;
  o->max_iter = 64;
  o->riemann_tol = 0.0;
  o->stream = nullptr;
  o->n_boxes = 1;
  o->box_cells = nullptr;
  o->box_faces = nullptr;
  o->entropy = 0;
  o->mach_thresh = 1.1;
  o->alpha_s = 0.01;
  o->regularize = 0;
  o->eta = 0.25;
  o->chi = 1.0;
}

const char* amm_last_error(const amm_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

int amm_create(amm_ctx** out, int dim, int64_t n, const double* gen, int64_t nf, const int32_t* cells,
               const int8_t* shift, const double* area, const double* cen, const double* box, const double* Q,
               double gamma, const amm_options* opt_in) {
  amm_ctx* c = nullptr;
  if (!out) return AMM_ERR_INVALID_ARG;
  *out = nullptr;
  amm_options opt;
  if (opt_in)
    opt = *opt_in;
  else
    amm_default_options(&opt);
  if (dim != 2 && dim != 3) return AMM_ERR_INVALID_ARG;
  if (n < 2 || n > (int64_t)1 << 30 || nf < 1 || nf > ((int64_t)1 << 30) - 1) return AMM_ERR_INVALID_ARG;
  if (!gen || !cells || !shift || !area || !cen || !box || !Q) return AMM_ERR_INVALID_ARG;
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return AMM_ERR_INVALID_ARG;
  if (opt.precision < AMM_FP64 || opt.precision > AMM_FP32_LEARNED) return AMM_ERR_INVALID_ARG;
  if (opt.mesh_motion < AMM_EULERIAN || opt.mesh_motion > AMM_EXPLICIT_W) return AMM_ERR_INVALID_ARG;
  if (opt.max_iter < 1 || opt.max_iter > 10000) return AMM_ERR_INVALID_ARG;
  if (opt.n_boxes < 1 || opt.n_boxes > (1 << 20)) return AMM_ERR_INVALID_ARG;
  if (opt.entropy != 0 && opt.entropy != 1) return AMM_ERR_INVALID_ARG;
  if (opt.regularize != 0 && opt.regularize != 1) return AMM_ERR_INVALID_ARG;
  if (opt.regularize && (opt.mesh_motion == AMM_EULERIAN || !(opt.eta > 0.0) || !(opt.chi >= 0.0) ||
                         !std::isfinite(opt.eta) || !std::isfinite(opt.chi)))
    return AMM_ERR_INVALID_ARG;
  if (opt.entropy && (!(opt.mach_thresh >= 0.0) || !(opt.alpha_s >= 0.0) || !std::isfinite(opt.alpha_s)))
    return AMM_ERR_INVALID_ARG;
  if (!(opt.riemann_tol > 0.0)) opt.riemann_tol = (opt.precision == AMM_FP64) ? 1e-12 : 1e-6;
  const int nb = (int)opt.n_boxes;
  std::vector<int64_t> bc(nb + 1), bf(nb + 1);
  if (nb == 1) {
    bc[0] = 0; bc[1] = n; bf[0] = 0; bf[1] = nf;
  } else {
    if (!opt.box_cells || !opt.box_faces) return AMM_ERR_INVALID_ARG;
    for (int b = 0; b <= nb; b++) {
      bc[b] = opt.box_cells[b];
      bf[b] = opt.box_faces[b];
    }
    if (bc[0] != 0 || bc[nb] != n || bf[0] != 0 || bf[nb] != nf) return AMM_ERR_INVALID_ARG;
    for (int b = 0; b < nb; b++)
      if (bc[b + 1] <= bc[b] + 1 || bf[b + 1] <= bf[b]) return AMM_ERR_INVALID_ARG;
  }
  const int nv = dim + 2;
  // host validation of the mesh and the state
  if (!finite_all(gen, (size_t)n * dim) || !finite_all(area, (size_t)nf) || !finite_all(cen, (size_t)nf * dim) ||
      !finite_all(Q, (size_t)n * nv) || !finite_all(box, (size_t)nb * dim))
    return AMM_ERR_INVALID_ARG;
  for (int b = 0; b < nb; b++) {
    for (int d = 0; d < dim; d++)
      if (!(box[b * dim + d] > 0.0)) return AMM_ERR_INVALID_ARG;
    for (int64_t i = bc[b]; i < bc[b + 1]; i++)
      for (int d = 0; d < dim; d++) {
        const double x = gen[i * dim + d];
        if (!(x >= 0.0 && x < box[b * dim + d])) return AMM_ERR_INVALID_ARG;
      }
    for (int64_t k = bf[b]; k < bf[b + 1]; k++) {
      const int64_t L = cells[2 * k], R = cells[2 * k + 1];
      if (L < bc[b] || L >= bc[b + 1] || R < bc[b] || R >= bc[b + 1]) return AMM_ERR_INVALID_ARG;
      if (!(area[k] >= 0.0)) return AMM_ERR_INVALID_ARG;
      bool zero = true;
      for (int d = 0; d < dim; d++) zero &= shift[k * dim + d] == 0;
      if (L == R && zero) return AMM_ERR_INVALID_ARG;
    }
  }
  for (int64_t i = 0; i < n; i++)
    if (!(Q[i * nv] > 0.0)) return AMM_ERR_NONPOSITIVE_STATE;

  c = new amm_ctx();
  c->dim = dim;
  c->n = n;
  c->nf = nf;
  c->nboxes = nb;
  c->gamma = gamma;
  c->opt = opt;
  c->box_cells = bc;
  c->box_faces = bf;
  c->nf_cap = nf;
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) {
    int rc = cuda_fail(c, e0, "cudaGetDevice");
    fprintf(stderr, "amm_create: %s\n", c->err.c_str());
    free_ctx(c);
    return rc;
  }
  auto bail = [&](int rc) {
    // keep the message on stderr: the context is gone
    if (rc != AMM_OK) fprintf(stderr, "amm_create: %s\n", c->err.c_str());
    free_ctx(c);
    return rc;
  };
#define CUB(call)                                    \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, #call)); \
  } while (0)
  if (opt.stream) {
    c->stream = (cudaStream_t)opt.stream;
  } else {
    CUB(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  CUB(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
  c->opt.stream = c->stream;

  // Internal numbering: cells of each box along a Morton (Z-order) curve of
  // their positions, faces by their new left cell, so that neighbouring cells
  // share cache lines in the gathers (the paper orders its points along a
  // space-filling curve for the same reason).  Every getter and setter maps
  // back to the caller's numbering.
  std::vector<int> perm(n), inv(n), fperm(nf);
  {
    std::vector<uint64_t> key(n);
    for (int b = 0; b < nb; b++) {
      for (int64_t i = bc[b]; i < bc[b + 1]; i++) {
        uint64_t k = 0;
        for (int d = 0; d < dim; d++) {
          const double x = gen[i * dim + d] / box[b * dim + d];
          uint64_t qd = (uint64_t)std::min(2097151.0, std::max(0.0, std::floor(x * 2097152.0)));
          for (int bit = 0; bit < 21; bit++) k |= ((qd >> bit) & 1ull) << (bit * dim + d);
        }
        key[i] = k;
      }
      for (int64_t i = bc[b]; i < bc[b + 1]; i++) perm[i] = (int)i;
      std::stable_sort(perm.begin() + bc[b], perm.begin() + bc[b + 1],
                       [&](int x, int y) { return key[x] < key[y]; });
    }
    for (int64_t i = 0; i < n; i++) inv[perm[i]] = (int)i;
    for (int64_t k = 0; k < nf; k++) fperm[k] = (int)k;
    for (int b = 0; b < nb; b++)
      std::stable_sort(fperm.begin() + bf[b], fperm.begin() + bf[b + 1], [&](int x, int y) {
        const int lx = inv[cells[2 * x]], ly = inv[cells[2 * y]];
        if (lx != ly) return lx < ly;
        return inv[cells[2 * x + 1]] < inv[cells[2 * y + 1]];
      });
  }
  std::vector<int2> lr_new(nf);
  for (int64_t k = 0; k < nf; k++)
    lr_new[k] = make_int2(inv[cells[2 * fperm[k]]], inv[cells[2 * fperm[k] + 1]]);
  // cell -> (face, side) lists, each cell's list ordered by the direction of
  // its outward normals (dominant axis and sign, then the signs of the other
  // two components, then larger faces first) so that the k-th entries of
  // neighbouring cells point the same way and their gathers share lines
  std::vector<int> off(n + 1, 0);
  for (int64_t k = 0; k < nf; k++) {
    off[lr_new[k].x + 1]++;
    off[lr_new[k].y + 1]++;
  }
  for (int64_t i = 0; i < n; i++) off[i + 1] += off[i];
  std::vector<int2> csr(2 * nf);
  {
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int64_t k = 0; k < nf; k++) {
      const int L = lr_new[k].x, R = lr_new[k].y;
      csr[fill[L]++] = make_int2((int)(k << 1), R);
      csr[fill[R]++] = make_int2((int)((k << 1) | 1), L);
    }
    std::vector<int> dkey(nf);   // direction class of the face normal L -> R
    std::vector<int> box_of_face(nf);
    for (int b = 0; b < nb; b++)
      for (int64_t k = bf[b]; k < bf[b + 1]; k++) box_of_face[k] = b;
    auto klass = [&](const double* d) {
      int ax = 0;
      for (int q = 1; q < dim; q++)
        if (std::fabs(d[q]) > std::fabs(d[ax])) ax = q;
      int cls = 2 * ax + (d[ax] < 0 ? 1 : 0);
      int sub = 0, bit = 0;
      for (int q = 0; q < dim; q++)
        if (q != ax) sub |= (d[q] < 0 ? 1 : 0) << (bit++);
      return cls * 4 + sub;
    };
    for (int64_t k = 0; k < nf; k++) {
      const int64_t o = fperm[k];
      const int b = box_of_face[o];
      double dl[3], dr[3];
      for (int d = 0; d < dim; d++) {
        const double x = gen[(int64_t)cells[2 * o + 1] * dim + d] + shift[o * dim + d] * box[b * dim + d] -
                         gen[(int64_t)cells[2 * o] * dim + d];
        dl[d] = x;
        dr[d] = -x;
      }
      dkey[k] = klass(dl) * 32 + klass(dr);  // both sides' classes, packed
    }
    for (int64_t i = 0; i < n; i++)
      std::stable_sort(csr.begin() + off[i], csr.begin() + off[i + 1], [&](const int2& x, const int2& y) {
        const int kx = x.x >> 1, ky = y.x >> 1;
        const int cx = (x.x & 1) ? dkey[kx] % 32 : dkey[kx] / 32;
        const int cy = (y.x & 1) ? dkey[ky] % 32 : dkey[ky] / 32;
        if (cx != cy) return cx < cy;
        return area[fperm[kx]] > area[fperm[ky]];
      });
  }
  int max_inc = 0;
  for (int64_t i = 0; i < n; i++) {
    if (off[i + 1] == off[i]) return bail(fail(c, AMM_ERR_OPEN_CELL, "a cell has no faces"));
    max_inc = std::max(max_inc, off[i + 1] - off[i]);
  }
  // bits reserved so that a cell's fixed-point flux sum cannot overflow
  c->headroom = 1;
  while ((1 << c->headroom) < max_inc + 1) c->headroom++;
  c->headroom += 1;
  // tiles
  std::vector<Tile> ct, ft;
  std::vector<int> bfc(nb + 1, 0);
  for (int b = 0; b < nb; b++) {
    bfc[b] = (int)ct.size();
    for (int64_t s = bc[b]; s < bc[b + 1]; s += amm::CELL_TILE)
      ct.push_back(Tile{b, (int)s, (int)std::min<int64_t>(s + amm::CELL_TILE, bc[b + 1]), 0});
    for (int64_t s = bf[b]; s < bf[b + 1]; s += amm::FACE_TILE)
      ft.push_back(Tile{b, (int)s, (int)std::min<int64_t>(s + amm::FACE_TILE, bf[b + 1]), 0});
  }
  bfc[nb] = (int)ct.size();
  c->n_ctiles = (int)ct.size();
  c->n_ftiles = (int)ft.size();
  c->box_first_ctile_h = bfc;
  // padded 3-vectors
  std::vector<double> gen3((size_t)n * 3, 0.0), cen3((size_t)nf * 3, 0.0), box3((size_t)nb * 3, 1.0);
  std::vector<int8_t> sh3((size_t)nf * 3, 0);
  std::vector<double> area_new(nf);
  for (int64_t i = 0; i < n; i++)
    for (int d = 0; d < dim; d++) gen3[i * 3 + d] = gen[(int64_t)perm[i] * dim + d];
  for (int64_t k = 0; k < nf; k++) {
    const int64_t o = fperm[k];
    area_new[k] = area[o];
    for (int d = 0; d < dim; d++) {
      cen3[k * 3 + d] = cen[o * dim + d];
      sh3[k * 3 + d] = shift[o * dim + d];
    }
  }
  for (int b = 0; b < nb; b++)
    for (int d = 0; d < dim; d++) box3[b * 3 + d] = box[b * dim + d];
  c->box_h = box3;

  const size_t rs = c->real_size();
  CUB(dalloc(&c->gen, (size_t)n * 3));
  CUB(dalloc(&c->box, (size_t)nb * 3));
  CUB(dalloc(&c->Q, (size_t)n * 5));
  CUB(dalloc(&c->lr, (size_t)nf));
  CUB(dalloc(&c->cell_perm, (size_t)n));
  CUB(dalloc(&c->face_perm, (size_t)nf));
  CUB(dalloc(&c->csr_off, (size_t)n + 1));
  CUB(dalloc(&c->csr, (size_t)2 * nf));
  CUB(dalloc(&c->ctiles, ct.size()));
  CUB(dalloc(&c->ftiles, ft.size()));
  CUB(dalloc(&c->box_first_ctile, (size_t)nb + 1));
  CUB(cudaMalloc(&c->fgeo, rs * 4 * 2 * (size_t)nf));
  CUB(cudaMalloc(&c->igAB, rs * 4 * 4 * (size_t)nf));
  CUB(dalloc(&c->cgeo64, (size_t)n));
  CUB(cudaMalloc(&c->cgeo, rs * 4 * (size_t)n));
  CUB(cudaMalloc(&c->crad, rs * (size_t)n));
  CUB(cudaMalloc(&c->cw, rs * 8 * (size_t)n));
  CUB(cudaMalloc(&c->grad, rs * 16 * (size_t)n));
  if (opt.mesh_motion == AMM_EULERIAN) {
    CUB(cudaMalloc(&c->cwp, rs * 8 * (size_t)n));
    if (opt.entropy) CUB(cudaMalloc(&c->Apw, rs * (size_t)n));
  }
  if (opt.mesh_motion == AMM_EXPLICIT_W) {
    CUB(cudaMalloc(&c->wmesh, rs * 4 * (size_t)n));
    CUB(cudaMemsetAsync(c->wmesh, 0, rs * 4 * (size_t)n, c->stream));
  }

  CUB(cudaMalloc(&c->flux, rs * 4 * (size_t)nf));
  CUB(cudaMalloc(&c->fluxE, rs * (size_t)nf));
  if (opt.regularize) {
    CUB(cudaMalloc(&c->wcorr, rs * 4 * (size_t)n));
    CUB(cudaMemsetAsync(c->wcorr, 0, rs * 4 * (size_t)n, c->stream));
  }
  if (opt.entropy) {
    CUB(dalloc(&c->S, (size_t)n));
    CUB(cudaMalloc(&c->Aw, rs * (size_t)n));
    CUB(cudaMalloc(&c->gradA, rs * 4 * (size_t)n));
    CUB(cudaMalloc(&c->fluxS, rs * (size_t)nf));
    CUB(cudaMalloc(&c->machf, rs * (size_t)nf));
    CUB(cudaMalloc(&c->ekmax, rs * (size_t)n));
    CUB(dalloc(&c->kept, (size_t)n));
    CUB(cudaMemsetAsync(c->ekmax, 0, rs * (size_t)n, c->stream));
    CUB(cudaMemsetAsync(c->kept, 0, (size_t)n, c->stream));
  }
  CUB(dalloc(&c->cour_bits, (size_t)nb));
  CUB(dalloc(&c->fmax_bits, (size_t)amm::FMAX_STRIDE * nb));
  CUB(cudaMemsetAsync(c->fmax_bits, 0, sizeof(unsigned) * amm::FMAX_STRIDE * nb, c->stream));
  CUB(dalloc(&c->dt_box, (size_t)nb));
  CUB(dalloc(&c->dt_used, (size_t)nb));
  CUB(dalloc(&c->partial, (size_t)5 * 8 * ct.size()));
  CUB(dalloc(&c->totals, (size_t)5 * nb));
  CUB(dalloc(&c->stats, 1));
  CUB(dalloc(&c->box_status, (size_t)nb));
  CUB(cudaMemsetAsync(c->box_status, 0, sizeof(unsigned) * nb, c->stream));
  CUB(dalloc(&c->closure, (size_t)n));
  CUB(dalloc(&c->counter, 4));
  CUB(dalloc(&c->barrier, 2));
  CUB(cudaMemsetAsync(c->barrier, 0, sizeof(unsigned) * 2, c->stream));
  CUB(cudaMemsetAsync(c->stats, 0, sizeof(amm::DeviceStats), c->stream));
  CUB(cudaMemsetAsync(c->dt_box, 0, sizeof(double) * nb, c->stream));
  CUB(cudaMemsetAsync(c->dt_used, 0, sizeof(double) * nb, c->stream));
  CUB(cudaMemsetAsync(c->cour_bits, 0xff, sizeof(unsigned long long) * nb, c->stream));
  CUB(cudaMemsetAsync(c->flux, 0, rs * 4 * (size_t)nf, c->stream));
  CUB(cudaMemsetAsync(c->fluxE, 0, rs * (size_t)nf, c->stream));
  CUB(cudaMemcpyAsync(c->gen, gen3.data(), sizeof(double) * gen3.size(), cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->box, box3.data(), sizeof(double) * box3.size(), cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->lr, lr_new.data(), sizeof(int2) * (size_t)nf, cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->cell_perm, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->face_perm, fperm.data(), sizeof(int) * (size_t)nf, cudaMemcpyHostToDevice, c->stream));
  c->perm_h = perm;
  CUB(cudaMemcpyAsync(c->csr_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->csr, csr.data(), sizeof(int2) * csr.size(), cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->ctiles, ct.data(), sizeof(Tile) * ct.size(), cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->ftiles, ft.data(), sizeof(Tile) * ft.size(), cudaMemcpyHostToDevice, c->stream));
  CUB(cudaMemcpyAsync(c->box_first_ctile, bfc.data(), sizeof(int) * bfc.size(), cudaMemcpyHostToDevice, c->stream));
  // face inputs through scratch: area [nf], centroid [nf][3], shift [nf][3]
  {
    double* d_area = nullptr;
    double* d_cen = nullptr;
    int8_t* d_sh = nullptr;
    CUB(dalloc(&d_area, (size_t)nf));
    CUB(dalloc(&d_cen, (size_t)nf * 3));
    CUB(dalloc(&d_sh, (size_t)nf * 3));
    CUB(cudaMemcpyAsync(d_area, area_new.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, c->stream));
    CUB(cudaMemcpyAsync(d_cen, cen3.data(), sizeof(double) * cen3.size(), cudaMemcpyHostToDevice, c->stream));
    CUB(cudaMemcpyAsync(d_sh, sh3.data(), sh3.size(), cudaMemcpyHostToDevice, c->stream));
    cudaError_t eg = amm::launch_face_geometry(c, d_area, d_cen, d_sh);
    cudaStreamSynchronize(c->stream);
    cudaFree(d_area);
    cudaFree(d_cen);
    cudaFree(d_sh);
    if (eg != cudaSuccess) return bail(cuda_fail(c, eg, "face/cell geometry"));
  }
  // closure and volume checks
  {
    std::vector<float> clo(n);
    std::vector<R4<double>> cg(n);
    CUB(cudaMemcpy(clo.data(), c->closure, sizeof(float) * n, cudaMemcpyDeviceToHost));
    CUB(cudaMemcpy(cg.data(), c->cgeo64, sizeof(R4<double>) * n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; i++) {
      if (!(cg[i].x > 0.0))
        return bail(fail(c, AMM_ERR_OPEN_CELL, "cell " + std::to_string(perm[i]) + " has volume <= 0"));
      if (!(clo[i] <= 1e-9f))
        return bail(fail(c, AMM_ERR_OPEN_CELL, "cell " + std::to_string(perm[i]) + " is not closed (relative closure " +
                                                   std::to_string(clo[i]) + ")"));
    }
  }
  *out = c;
  const int rc = amm_set_state(c, Q);
  if (rc != AMM_OK) {
    *out = nullptr;
    return bail(rc);
  }
#undef CUB
  return AMM_OK;
}

int amm_create_device(amm_ctx** out, int dim, int64_t n, const double* gen_d, int64_t nf, const int32_t* cells_d,
                      const int8_t* shift_d, const double* area_d, const double* cen_d, const double* box,
                      const double* Q_d, double gamma, const amm_options* opt) {
  if (!out) return AMM_ERR_INVALID_ARG;
  *out = nullptr;
  if ((dim != 2 && dim != 3) || n < 2 || n > (int64_t)1 << 30 || nf < 1 || nf > ((int64_t)1 << 30) - 1)
    return AMM_ERR_INVALID_ARG;
  if (!gen_d || !cells_d || !shift_d || !area_d || !cen_d || !box || !Q_d) return AMM_ERR_INVALID_ARG;
  std::vector<double> gen((size_t)n * dim), area((size_t)nf), cen((size_t)nf * dim), Q((size_t)n * (dim + 2));
  std::vector<int32_t> cells((size_t)nf * 2);
  std::vector<int8_t> shift((size_t)nf * dim);
  const struct {
    void* dst;
    const void* src;
    size_t bytes;
  } copies[] = {{gen.data(), gen_d, sizeof(double) * gen.size()},     {cells.data(), cells_d, sizeof(int32_t) * cells.size()},
                {shift.data(), shift_d, shift.size()},                 {area.data(), area_d, sizeof(double) * area.size()},
                {cen.data(), cen_d, sizeof(double) * cen.size()},      {Q.data(), Q_d, sizeof(double) * Q.size()}};
  for (const auto& cp : copies)
    if (cudaMemcpy(cp.dst, cp.src, cp.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return AMM_ERR_CUDA;
    }
  return amm_create(out, dim, n, gen.data(), nf, cells.data(), shift.data(), area.data(), cen.data(), box, Q.data(),
                    gamma, opt);
}

int amm_destroy(amm_ctx* c) {
  if (!c) return AMM_OK;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
  return AMM_OK;
}

static int set_state_common(amm_ctx* c, const double* Qdev_aos) {
  CU(cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), c->stream));
  CU(dispatch(c, [&] { return amm::launch_set_state<double>(c, Qdev_aos, c->counter); },
              [&] { return amm::launch_set_state<float>(c, Qdev_aos, c->counter); }));
  unsigned long long bad = 0;
  CU(cudaMemcpyAsync(&bad, c->counter, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->grads_fresh = false;
  c->totals_fresh = false;
  if (bad) return fail(c, AMM_ERR_NONPOSITIVE_STATE, std::to_string(bad) + " cells with m <= 0 or P <= 0");
  return AMM_OK;
}

int amm_set_state(amm_ctx* c, const double* Q) {
  if (!c || !Q) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  const size_t cnt = (size_t)c->n * (c->dim + 2);
  CU(ensure_scratch(c, cnt));
  CU(cudaMemcpyAsync(c->scratch, Q, sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream));
  return set_state_common(c, c->scratch);
}

int amm_set_state_device(amm_ctx* c, const double* Qd) {
  if (!c || !Qd) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  return set_state_common(c, Qd);
}

int amm_set_mesh_velocity(amm_ctx* c, const double* w) {
  if (!c || !w) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  if (c->opt.mesh_motion != AMM_EXPLICIT_W) return fail(c, AMM_ERR_INVALID_ARG, "mesh motion is not explicit");
  const size_t cnt = (size_t)c->n * c->dim;
  if (!finite_all(w, cnt)) return fail(c, AMM_ERR_INVALID_ARG, "non-finite mesh velocity");
  CU(ensure_scratch(c, std::max(cnt, (size_t)c->n * (c->dim + 2))));
  CU(cudaMemcpyAsync(c->scratch, w, sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream));
  CU(dispatch(c, [&] { return amm::launch_set_wmesh<double>(c, c->scratch); },
              [&] { return amm::launch_set_wmesh<float>(c, c->scratch); }));
  CU(cudaStreamSynchronize(c->stream));
  c->grads_fresh = false;
  return AMM_OK;
}

int amm_gradients(amm_ctx* c) {
  if (!c) return AMM_ERR_INVALID_ARG;
  CU(run_gradients(c, 0.0));
  c->grads_fresh = true;
  return AMM_OK;
}

int amm_timestep(amm_ctx* c, double cfl, double* dt_out) {
  if (!c || !dt_out || !(cfl > 0.0)) return fail(c, AMM_ERR_INVALID_ARG, "bad argument");
  // the Courant minimum of the current state (and the regularity-corrected
  // mesh velocities, which the drift takes)
  CU(dispatch(c, [&] { return amm::launch_courant<double>(c); }, [&] { return amm::launch_courant<float>(c); }));
  std::vector<unsigned long long> bits(c->nboxes);
  CU(cudaMemcpyAsync(bits.data(), c->cour_bits, sizeof(unsigned long long) * c->nboxes, cudaMemcpyDeviceToHost,
                     c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int b = 0; b < c->nboxes; b++) {
    double t;
    std::memcpy(&t, &bits[b], sizeof t);
    dt_out[b] = cfl * t;
  }
  return AMM_OK;
}

static int step_with_dt_box(amm_ctx* c) {
  if (c->opt.precision == AMM_FP32_LEARNED && !c->mlp_loaded)
    return fail(c, AMM_ERR_NOT_READY, "no proposal weights loaded");
  CU(run_gradients(c, 0.0));   // always: the static mesh's predicted records take this dt
  CU(run_step_tail(c, 0.0));
  c->grads_fresh = false;
  c->totals_fresh = true;
  c->have_step = true;
  return AMM_OK;
}

int amm_step(amm_ctx* c, double dt) {
  if (!c || !(dt >= 0.0) || !std::isfinite(dt)) return fail(c, AMM_ERR_INVALID_ARG, "bad time step");
  std::vector<double> d(c->nboxes, dt);
  CU(cudaMemcpyAsync(c->dt_box, d.data(), sizeof(double) * c->nboxes, cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));  // the host vector goes out of scope
  return step_with_dt_box(c);
}

int amm_step_boxes(amm_ctx* c, const double* dt) {
  if (!c || !dt) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  for (int b = 0; b < c->nboxes; b++)
    if (!(dt[b] >= 0.0) || !std::isfinite(dt[b])) return fail(c, AMM_ERR_INVALID_ARG, "bad time step");
  CU(cudaMemcpyAsync(c->dt_box, dt, sizeof(double) * c->nboxes, cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return step_with_dt_box(c);
}

int amm_advance(amm_ctx* c, double cfl, int64_t nsteps, int use_graph) {
  if (!c || !(cfl > 0.0) || nsteps < 0) return fail(c, AMM_ERR_INVALID_ARG, "bad argument");
  if (c->opt.precision == AMM_FP32_LEARNED && !c->mlp_loaded)
    return fail(c, AMM_ERR_NOT_READY, "no proposal weights loaded");
  if (nsteps == 0) return AMM_OK;
  const bool pers = c->persistent != 0;
  auto one_step = [&]() -> cudaError_t {
    if (pers) {
      cudaError_t e = mark(c, 0);
      if (e == cudaSuccess) {
        if (c->opt.precision == AMM_FP32_LEARNED)
          e = amm::launch_step_persistent_learned(c, cfl);
        else
          e = dispatch(c, [&] { return amm::launch_step_persistent<double>(c, cfl); },
                       [&] { return amm::launch_step_persistent<float>(c, cfl); });
      }
      if (e == cudaSuccess) e = mark(c, 1);
      if (e == cudaSuccess) e = mark(c, 2);
      if (e == cudaSuccess) e = mark(c, 3);
      if (e == cudaSuccess) e = mark(c, 4);
      return e;
    }
    cudaError_t e = run_gradients(c, cfl);
    if (e == cudaSuccess) e = run_step_tail(c, cfl);
    return e;
  };
  if (!use_graph) {
    for (int64_t s = 0; s < nsteps; s++) CU(one_step());
  } else {
    if (!c->graph || c->graph_cfl != cfl || c->graph_profiled != c->profiling || c->graph_persistent != pers) {
      if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
      }
      // capture one whole step on the auxiliary stream
      CU(cudaStreamSynchronize(c->stream));
      cudaStream_t keep = c->stream;
      c->stream = c->aux_stream;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e1 = one_step();
        e = cudaStreamEndCapture(c->stream, &g);
        if (e == cudaSuccess) e = e1;
      }
      c->stream = keep;
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e, "step graph capture");
      }
      e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
      c->graph_cfl = cfl;
      c->graph_profiled = c->profiling;
      c->graph_persistent = pers;
    }
    for (int64_t s = 0; s < nsteps; s++) CU(cudaGraphLaunch(c->graph, c->stream));
  }
  c->grads_fresh = false;
  c->totals_fresh = true;
  c->have_step = true;
  return AMM_OK;
}

// Buffers and the leaf-bucket order of the cells for individual time steps,
// once per context (the mesh is static): a uniform grid of 2^L buckets per
// axis over the box with L = floor(log2(n^(1/dim) / 2)) (about 2^dim cells per
// bucket on a lattice), at least 1 and at most 7 (3D) or 9 (2D) levels below
// the root.
static int individual_setup(amm_ctx* c) {
  const int64_t n = c->n;
  const int dim = c->dim;
  int L = (int)std::floor(std::log2(std::pow((double)n, 1.0 / dim) / 2.0));
  L = std::max(1, std::min(L, dim == 3 ? 7 : 9));
  c->ind_levels = L + 1;
  c->ind_level_off_h.assign(c->ind_levels + 1, 0);
  for (int l = 0; l < c->ind_levels; l++)
    c->ind_level_off_h[l + 1] = c->ind_level_off_h[l] + (1 << (dim * l));
  const int leaves = 1 << (dim * L);
  const int side = 1 << L;
  std::vector<double> g((size_t)n * 3);
  CU(cudaMemcpy(g.data(), c->gen, sizeof(double) * g.size(), cudaMemcpyDeviceToHost));
  std::vector<int> bucket((size_t)n), off((size_t)leaves + 1, 0), slot_cell((size_t)n), cell_slot((size_t)n);
  for (int64_t i = 0; i < n; i++) {
    int ib[3] = {0, 0, 0};
    for (int a = 0; a < dim; a++) {
      const double L_a = c->box_h[a];
      int q = (int)std::floor(g[3 * i + a] / L_a * side);
      ib[a] = std::max(0, std::min(side - 1, q));
    }
    bucket[i] = (dim == 3) ? (ib[0] * side + ib[1]) * side + ib[2] : ib[0] * side + ib[1];
    off[bucket[i] + 1]++;
  }
  for (int b = 0; b < leaves; b++) off[b + 1] += off[b];
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int64_t i = 0; i < n; i++) {
    const int s = fill[bucket[i]]++;
    slot_cell[s] = (int)i;
    cell_slot[i] = s;
  }
  CU(dalloc(&c->ind_bin, n));
  CU(dalloc(&c->ind_act, n));
  CU(dalloc(&c->ind_list, n));
  CU(dalloc(&c->ind_flist, c->nf_cap));
  CU(dalloc(&c->ind_count, 4));
  CU(dalloc(&c->ind_fstamp, c->nf_cap));
  CU(dalloc(&c->ind_cstamp, n));
  CU(dalloc(&c->ind_fdt, c->nf_cap));
  CU(dalloc(&c->ind_hist, 64));
  CU(dalloc(&c->ind_slot_cell, n));
  CU(dalloc(&c->ind_cell_slot, n));
  CU(dalloc(&c->ind_leaf_off, (size_t)leaves + 1));
  CU(dalloc(&c->ind_level_off, (size_t)c->ind_levels + 1));
  CU(dalloc((double4**)&c->ind_rec, 2 * (size_t)n));
  CU(dalloc((float4**)&c->ind_rec32, 2 * (size_t)n));
  CU(dalloc(&c->ind_loop, 1));
  CU(dalloc((float2**)&c->ind_node, (size_t)c->ind_level_off_h[c->ind_levels]));
  CU(cudaMemcpy(c->ind_slot_cell, slot_cell.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->ind_cell_slot, cell_slot.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->ind_leaf_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->ind_level_off, c->ind_level_off_h.data(), sizeof(int) * c->ind_level_off_h.size(),
                cudaMemcpyHostToDevice));
  CU(cudaMemset(c->ind_fstamp, 0xff, sizeof(int) * c->nf_cap));
  CU(cudaMemset(c->ind_cstamp, 0xff, sizeof(int) * n));
  c->ind_stamp = 0;
  c->ind_ready = true;
  return AMM_OK;
}

int amm_advance_individual(amm_ctx* c, double cfl, double dt_max, int max_depth, int signal_speed,
                           amm_cycle_stats* stats) {
  if (!c || !(cfl > 0.0) || !(dt_max > 0.0) || !std::isfinite(dt_max) || max_depth < 1 || max_depth > 40)
    return fail(c, AMM_ERR_INVALID_ARG, "bad argument");
  if (c->opt.mesh_motion != AMM_EULERIAN || c->nboxes != 1 || c->opt.entropy ||
      c->opt.precision == AMM_FP32_LEARNED)
    return fail(c, AMM_ERR_INVALID_ARG,
                "individual time steps need a static mesh (AMM_EULERIAN), one box, no entropy switch and the "
                "FP64 or FP32 form");
  if (!c->ind_ready) {
    const int rc = individual_setup(c);
    if (rc != AMM_OK) return rc;
  }
  const int64_t n = c->n;
  std::vector<unsigned> hist(64, 0u);
  hist[0] = (unsigned)n;
  CU(cudaMemsetAsync(c->ind_bin, 0, n, c->stream));
  CU(cudaMemsetAsync(c->ind_count, 0, sizeof(int) * 4, c->stream));
  CU(cudaMemcpyAsync(c->ind_hist, hist.data(), sizeof(unsigned) * 64, cudaMemcpyHostToDevice, c->stream));
  amm::IndLoop L0;
  std::memset(&L0, 0, sizeof L0);
  L0.T = 1ll << max_depth;
  L0.stamp = ++c->ind_stamp;
  L0.max_substeps = 1ull << 20;
  CU(cudaMemcpyAsync(c->ind_loop, &L0, sizeof L0, cudaMemcpyHostToDevice, c->stream));
  amm::IndView d;
  d.n = (int)n;
  d.nf = (int)c->nf;
  d.dim = c->dim;
  d.depth = max_depth;
  d.levels = c->ind_levels;
  d.signal = signal_speed ? 1 : 0;
  d.cfl = cfl;
  d.dtick = dt_max / (double)(1ll << max_depth);
  d.gamma = c->gamma;
  for (int a = 0; a < 3; a++) d.box[a] = c->box_h[a];
  d.gen = c->gen;
  d.loop = c->ind_loop;
  d.handle = 0;
  d.in_graph = 0;
  d.bin = c->ind_bin;
  d.act = c->ind_act;
  d.list = c->ind_list;
  d.flist = c->ind_flist;
  d.count = c->ind_count;
  d.fstamp = c->ind_fstamp;
  d.cstamp = c->ind_cstamp;
  d.fdt = c->ind_fdt;
  d.hist = c->ind_hist;
  d.slot_cell = c->ind_slot_cell;
  d.cell_slot = c->ind_cell_slot;
  d.leaf_off = c->ind_leaf_off;
  d.stats = c->stats;
  d.rec = (double4*)c->ind_rec;
  d.rec32 = (float4*)c->ind_rec32;
  d.node = (float2*)c->ind_node;
  d.level_off = c->ind_level_off;
  auto one_tick = [&]() -> cudaError_t {
    cudaError_t e = dispatch(c, [&] { return amm::launch_individual_tick<double>(c, d); },
                             [&] { return amm::launch_individual_tick<float>(c, d); });
    return e == cudaSuccess ? amm::launch_individual_next(c, d) : e;
  };
  amm::IndLoop L;
  if (c->ind_host_loop) {
    // one launch sequence and one synchronisation per tick
    do {
      CU(one_tick());
      CU(cudaMemcpyAsync(&L, c->ind_loop, sizeof L, cudaMemcpyDeviceToHost, c->stream));
      CU(cudaStreamSynchronize(c->stream));
    } while (L.go);
  } else {
    const double key[4] = {cfl, dt_max, (double)max_depth, signal_speed ? 1.0 : 0.0};
    if (!c->ind_exec || std::memcmp(key, c->ind_key, sizeof key) != 0) {
      // the cycle as one graph: a while node whose body is one tick, the
      // last kernel of which sets the condition
      if (c->ind_exec) cudaGraphExecDestroy(c->ind_exec);
      if (c->ind_graph) cudaGraphDestroy(c->ind_graph);
      c->ind_exec = nullptr;
      c->ind_graph = nullptr;
      CU(cudaGraphCreate(&c->ind_graph, 0));
      cudaGraphConditionalHandle h;
      CU(cudaGraphConditionalHandleCreate(&h, c->ind_graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      CU(cudaGraphAddNode(&node, c->ind_graph, nullptr, nullptr, 0, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      d.handle = h;
      d.in_graph = 1;
      CU(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      const cudaError_t e = one_tick();
      cudaGraph_t captured = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(c->stream, &captured);
      if (e != cudaSuccess) return cuda_fail(c, e, "capture of one tick");
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
      CU(cudaGraphInstantiate(&c->ind_exec, c->ind_graph, 0));
      std::memcpy(c->ind_key, key, sizeof key);
    }
    CU(cudaGraphLaunch(c->ind_exec, c->stream));
    CU(cudaMemcpyAsync(&L, c->ind_loop, sizeof L, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  c->ind_stamp = L.stamp;
  {
    const int rc = check_status(c);
    if (rc != AMM_OK) return rc;
  }
  amm_cycle_stats st;
  std::memset(&st, 0, sizeof st);
  st.substeps = (int64_t)L.substeps;
  st.face_fluxes = (int64_t)L.face_fluxes;
  st.activations = (int64_t)L.activations;
  st.deepest_bin = L.deepest;
  // every cell has finished its last step: fresh primitives of the new state
  CU(dispatch(c, [&] { return amm::launch_primitives<double>(c); },
              [&] { return amm::launch_primitives<float>(c); }));
  c->grads_fresh = false;
  c->totals_fresh = false;
  c->have_step = true;
  if (stats) *stats = st;
  CU(cudaStreamSynchronize(c->stream));
  return AMM_OK;
}

int amm_individual_host_loop(amm_ctx* c, int enable) {
  if (!c) return AMM_ERR_INVALID_ARG;
  c->ind_host_loop = enable != 0;
  return AMM_OK;
}

int amm_get_bins(amm_ctx* c, int32_t* bins) {
  if (!c || !bins) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  if (!c->ind_ready) return fail(c, AMM_ERR_NOT_READY, "no cycle of individual time steps yet");
  std::vector<signed char> b((size_t)c->n);
  CU(cudaMemcpyAsync(b.data(), c->ind_bin, c->n, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < c->n; i++) bins[c->perm_h[i]] = b[i];
  return AMM_OK;
}

int amm_harvest(amm_ctx* c, double cfl, float* states_device) {
  if (!c || !(cfl > 0.0) || !states_device) return fail(c, AMM_ERR_INVALID_ARG, "bad argument");
  if (c->opt.precision == AMM_FP64) return fail(c, AMM_ERR_INVALID_ARG, "harvest needs an FP32 form");
  if (c->opt.precision == AMM_FP32_LEARNED && !c->mlp_loaded)
    return fail(c, AMM_ERR_NOT_READY, "no proposal weights loaded");
  c->harvest = states_device;
  cudaError_t e = run_gradients(c, cfl);
  if (e == cudaSuccess) e = run_step_tail(c, cfl);
  c->harvest = nullptr;
  if (e != cudaSuccess) return cuda_fail(c, e, "harvest step");
  c->grads_fresh = false;
  c->totals_fresh = true;
  c->have_step = true;
  return AMM_OK;
}

int amm_drift(amm_ctx* c, double dt) {
  if (!c || !std::isfinite(dt)) return fail(c, AMM_ERR_INVALID_ARG, "bad argument");
  CU(amm::launch_drift(c, dt));
  return AMM_OK;
}

int amm_sync(amm_ctx* c) {
  if (!c) return AMM_ERR_INVALID_ARG;
  CU(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

int amm_get_state(amm_ctx* c, double* Q) {
  if (!c || !Q) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  const size_t cnt = (size_t)c->n * (c->dim + 2);
  CU(ensure_scratch(c, cnt));
  CU(dispatch(c, [&] { return amm::launch_get_state<double>(c, c->scratch); },
              [&] { return amm::launch_get_state<float>(c, c->scratch); }));
  CU(cudaMemcpyAsync(Q, c->scratch, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

int amm_get_state_device(amm_ctx* c, double* Qd) {
  if (!c || !Qd) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  CU(dispatch(c, [&] { return amm::launch_get_state<double>(c, Qd); },
              [&] { return amm::launch_get_state<float>(c, Qd); }));
  CU(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

int amm_get_primitives(amm_ctx* c, double* W) {
  if (!c || !W) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  const size_t cnt = (size_t)c->n * (c->dim + 2);
  CU(ensure_scratch(c, cnt));
  CU(dispatch(c, [&] { return amm::launch_get_primitives<double>(c, c->scratch); },
              [&] { return amm::launch_get_primitives<float>(c, c->scratch); }));
  CU(cudaMemcpyAsync(W, c->scratch, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return AMM_OK;
}

int amm_get_gradients(amm_ctx* c, double* g) {
  if (!c || !g) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  if (!c->grads_fresh) {
    CU(run_gradients(c, 0.0));
    c->grads_fresh = true;
  }
  const size_t cnt = (size_t)c->n * (c->dim + 2) * c->dim;
  CU(ensure_scratch(c, cnt));
  CU(dispatch(c, [&] { return amm::launch_get_gradients<double>(c, c->scratch); },
              [&] { return amm::launch_get_gradients<float>(c, c->scratch); }));
  CU(cudaMemcpyAsync(g, c->scratch, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return AMM_OK;
}

int amm_get_face_flux(amm_ctx* c, double* F) {
  if (!c || !F) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  const size_t cnt = (size_t)c->nf * (c->dim + 2);
  CU(ensure_scratch(c, cnt));
  CU(dispatch(c, [&] { return amm::launch_get_flux<double>(c, c->scratch); },
              [&] { return amm::launch_get_flux<float>(c, c->scratch); }));
  CU(cudaMemcpyAsync(F, c->scratch, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return AMM_OK;
}

int amm_get_geometry(amm_ctx* c, double* V, double* s) {
  if (!c || !V || !s) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  std::vector<R4<double>> cg(c->n);
  std::vector<double> g3((size_t)c->n * 3);
  CU(cudaMemcpyAsync(cg.data(), c->cgeo64, sizeof(R4<double>) * c->n, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(g3.data(), c->gen, sizeof(double) * g3.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < c->n; i++) {
    const int64_t o = c->perm_h[i];
    V[o] = cg[i].x;
    const double ds[3] = {cg[i].y, cg[i].z, cg[i].w};
    for (int d = 0; d < c->dim; d++) s[o * c->dim + d] = g3[i * 3 + d] + ds[d];
  }
  return AMM_OK;
}

int amm_get_totals(amm_ctx* c, double* tot) {
  if (!c || !tot) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  if (!c->totals_fresh) {
    CU(dispatch(c, [&] { return amm::launch_finish<double>(c, -1.0); },
                [&] { return amm::launch_finish<float>(c, -1.0); }));
    c->totals_fresh = true;
  }
  std::vector<double> t((size_t)5 * c->nboxes);
  CU(cudaMemcpyAsync(t.data(), c->totals, sizeof(double) * t.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const int nv = c->dim + 2;
  for (int b = 0; b < c->nboxes; b++) {
    tot[b * nv] = t[5 * b];
    tot[b * nv + 1] = t[5 * b + 1];
    tot[b * nv + 2] = t[5 * b + 2];
    if (c->dim == 3) tot[b * nv + 3] = t[5 * b + 3];
    tot[b * nv + c->dim + 1] = t[5 * b + 4];
  }
  return AMM_OK;
}

int amm_get_dt(amm_ctx* c, double* dt) {
  if (!c || !dt) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  CU(cudaMemcpyAsync(dt, c->dt_used, sizeof(double) * c->nboxes, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return AMM_OK;
}

int amm_get_generators(amm_ctx* c, double* gen) {
  if (!c || !gen) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  std::vector<double> g3((size_t)c->n * 3);
  CU(cudaMemcpyAsync(g3.data(), c->gen, sizeof(double) * g3.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < c->n; i++)
    for (int d = 0; d < c->dim; d++) gen[(int64_t)c->perm_h[i] * c->dim + d] = g3[i * 3 + d];
  return AMM_OK;
}

int amm_get_entropy(amm_ctx* c, double* S, uint8_t* kept) {
  if (!c || !S) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  if (!c->opt.entropy) return fail(c, AMM_ERR_INVALID_ARG, "the context has no entropy switch");
  std::vector<double> s((size_t)c->n);
  std::vector<unsigned char> k((size_t)c->n);
  CU(cudaMemcpyAsync(s.data(), c->S, sizeof(double) * s.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(k.data(), c->kept, k.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < c->n; i++) {
    S[c->perm_h[i]] = s[i];
    if (kept) kept[c->perm_h[i]] = k[i];
  }
  return check_status(c);
}

int amm_set_entropy(amm_ctx* c, const double* S) {
  if (!c || !S) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  if (!c->opt.entropy) return fail(c, AMM_ERR_INVALID_ARG, "the context has no entropy switch");
  std::vector<double> s((size_t)c->n);
  for (int64_t i = 0; i < c->n; i++) {
    s[i] = S[c->perm_h[i]];
    if (!(s[i] > 0.0) || !std::isfinite(s[i])) return fail(c, AMM_ERR_INVALID_ARG, "entropy must be positive");
  }
  CU(cudaMemcpyAsync(c->S, s.data(), sizeof(double) * s.size(), cudaMemcpyHostToDevice, c->stream));
  CU(dispatch(c, [&] { return amm::launch_primitives<double>(c); }, [&] { return amm::launch_primitives<float>(c); }));
  CU(cudaStreamSynchronize(c->stream));
  c->grads_fresh = false;
  return AMM_OK;
}

int amm_get_stats(amm_ctx* c, amm_stats* s) {
  if (!c || !s) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  amm::DeviceStats d;
  CU(cudaMemcpyAsync(&d, c->stats, sizeof(d), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  std::memset(s, 0, sizeof(*s));
  s->steps = (int64_t)d.steps;
  s->faces = (int64_t)d.faces;
  s->newton_iters = (int64_t)d.newton_iters;
  s->newton_fail = (int64_t)d.newton_fail;
  s->fallback_faces = (int64_t)d.fallback;
  s->vacuum_faces = (int64_t)d.vacuum;
  s->guard_faces = (int64_t)d.guard;
  s->nonpositive_cells = (int64_t)d.nonpos;
  s->newton_max = (int32_t)d.newton_max;
  s->status = d.status;
  for (int b = 0; b < 16; b++) s->newton_hist[b] = (int64_t)d.hist[b];
  s->entropy_kept = (int64_t)d.kept;
  return AMM_OK;
}

int amm_profile(amm_ctx* c, int enable) {
  if (!c) return AMM_ERR_INVALID_ARG;
  if (enable && !c->prof_ev[0])
    for (cudaEvent_t& ev : c->prof_ev) CU(cudaEventCreate(&ev));
  c->profiling = enable != 0;
  return AMM_OK;
}

int amm_get_kernel_times(amm_ctx* c, float* ms) {
  if (!c || !ms) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  if (!c->profiling) return fail(c, AMM_ERR_NOT_READY, "profiling is off");
  CU(cudaEventSynchronize(c->prof_ev[4]));
  for (int k = 0; k < 4; k++) CU(cudaEventElapsedTime(&ms[k], c->prof_ev[k], c->prof_ev[k + 1]));
  return AMM_OK;
}

int amm_set_tuning(amm_ctx* c, const amm_tuning* t) {
  if (!c || !t) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  auto ok_lanes = [](int g) { return g == 1 || g == 2 || g == 4 || g == 8; };
  if (!ok_lanes(t->grad_lanes) || !ok_lanes(t->update_lanes) || (t->flux_block != 128 && t->flux_block != 256))
    return fail(c, AMM_ERR_INVALID_ARG, "tuning values out of range");
  if (t->persistent != 0 && t->persistent != 1) return fail(c, AMM_ERR_INVALID_ARG, "persistent must be 0 or 1");
  c->grad_lanes = t->grad_lanes;
  c->update_lanes = t->update_lanes;
  c->flux_block = t->flux_block;
  c->persistent = t->persistent;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return AMM_OK;
}

int amm_get_tuning(amm_ctx* c, amm_tuning* t) {
  if (!c || !t) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  t->grad_lanes = c->grad_lanes;
  t->update_lanes = c->update_lanes;
  t->flux_block = c->flux_block;
  t->persistent = c->persistent;
  t->step_ms = c->tuned_ms;
  return AMM_OK;
}

int amm_autotune(amm_ctx* c, double cfl, int reps, amm_tuning* out) {
  if (!c || !(cfl > 0.0) || reps < 1) return fail(c, AMM_ERR_INVALID_ARG, "bad argument");
  if (c->opt.precision == AMM_FP32_LEARNED && !c->mlp_loaded)
    return fail(c, AMM_ERR_NOT_READY, "no proposal weights loaded");
  // keep the state: the trial steps run from the same input
  const size_t qn = (size_t)c->n * 5;
  double* saved = nullptr;
  CU(cudaMalloc((void**)&saved, sizeof(double) * qn));
  CU(cudaMemcpyAsync(saved, c->Q, sizeof(double) * qn, cudaMemcpyDeviceToDevice, c->stream));
  const bool prof = c->profiling;
  int rc = amm_profile(c, 1);
  static const int lanes[4] = {1, 2, 4, 8};
  static const int blocks[2] = {128, 256};
  float best[3] = {1e30f, 1e30f, 1e30f};
  int pick[3] = {c->grad_lanes, c->update_lanes, c->flux_block};
  for (int v = 0; v < 4 && rc == AMM_OK; v++) {
    amm_tuning t{lanes[v], lanes[v], blocks[v % 2], 0, 0.f};
    rc = amm_set_tuning(c, &t);
    std::vector<float> g, f, u;
    for (int r = 0; r < reps + 1 && rc == AMM_OK; r++) {
      cudaError_t e = cudaMemcpyAsync(c->Q, saved, sizeof(double) * qn, cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess)
        e = dispatch(c, [&] { return amm::launch_primitives<double>(c); },
                     [&] { return amm::launch_primitives<float>(c); });
      if (e != cudaSuccess) {
        rc = cuda_fail(c, e, "autotune reset");
        break;
      }
      e = run_gradients(c, cfl);
      if (e == cudaSuccess) e = run_step_tail(c, cfl);
      if (e != cudaSuccess) {
        rc = cuda_fail(c, e, "autotune step");
        break;
      }
      float ms[4];
      rc = amm_get_kernel_times(c, ms);
      if (r > 0) {  // the first trial warms up
        g.push_back(ms[0]);
        f.push_back(ms[1]);
        u.push_back(ms[2]);
      }
    }
    if (rc != AMM_OK) break;
    auto med = [](std::vector<float> x) {
      std::sort(x.begin(), x.end());
      return x[x.size() / 2];
    };
    const float mg = med(g), mf = med(f), mu = med(u);
    if (mg < best[0]) { best[0] = mg; pick[0] = lanes[v]; }
    if (mu < best[2]) { best[2] = mu; pick[1] = lanes[v]; }
    if (mf < best[1]) { best[1] = mf; pick[2] = blocks[v % 2]; }
  }
  cudaMemcpyAsync(c->Q, saved, sizeof(double) * qn, cudaMemcpyDeviceToDevice, c->stream);
  dispatch(c, [&] { return amm::launch_primitives<double>(c); }, [&] { return amm::launch_primitives<float>(c); });
  cudaStreamSynchronize(c->stream);
  cudaFree(saved);
  amm_profile(c, prof ? 1 : 0);
  cudaMemsetAsync(c->stats, 0, sizeof(amm::DeviceStats), c->stream);
  c->grads_fresh = false;
  c->totals_fresh = false;
  if (rc != AMM_OK) return rc;
  amm_tuning t{pick[0], pick[1], pick[2], 0, best[0] + best[1] + best[2]};
  rc = amm_set_tuning(c, &t);
  // then the whole step: the tuned kernel sequence against one persistent
  // launch (event-timed full steps from the same state)
  if (rc == AMM_OK) {
    float best_ms[2] = {1e30f, 1e30f};
    cudaEvent_t e0, e1;
    CU(cudaMalloc((void**)&saved, sizeof(double) * qn));
    CU(cudaMemcpyAsync(saved, c->Q, sizeof(double) * qn, cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (int pm = 0; pm < 2 && rc == AMM_OK; pm++) {
      c->persistent = pm;
      for (int r = 0; r < reps + 1 && rc == AMM_OK; r++) {
        cudaMemcpyAsync(c->Q, saved, sizeof(double) * qn, cudaMemcpyDeviceToDevice, c->stream);
        dispatch(c, [&] { return amm::launch_primitives<double>(c); }, [&] { return amm::launch_primitives<float>(c); });
        cudaEventRecord(e0, c->stream);
        rc = amm_advance(c, cfl, 1, 0);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best_ms[pm]) best_ms[pm] = ms;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(c->Q, saved, sizeof(double) * qn, cudaMemcpyDeviceToDevice, c->stream);
    dispatch(c, [&] { return amm::launch_primitives<double>(c); }, [&] { return amm::launch_primitives<float>(c); });
    cudaStreamSynchronize(c->stream);
    cudaFree(saved);
    cudaMemsetAsync(c->stats, 0, sizeof(amm::DeviceStats), c->stream);
    c->grads_fresh = false;
    c->totals_fresh = false;
    c->have_step = false;
    t.persistent = best_ms[1] < best_ms[0] ? 1 : 0;
    c->persistent = t.persistent;
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
  }
  c->tuned_ms = t.step_ms;
  if (out) *out = t;
  return rc;
}

int amm_get_box_status(amm_ctx* c, uint32_t* status) {
  if (!c || !status) return fail(c, AMM_ERR_INVALID_ARG, "null argument");
  CU(cudaMemcpyAsync(status, c->box_status, sizeof(unsigned) * c->nboxes, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return AMM_OK;
}

int amm_reset_stats(amm_ctx* c) {
  if (!c) return AMM_ERR_INVALID_ARG;
  CU(cudaMemsetAsync(c->box_status, 0, sizeof(unsigned) * c->nboxes, c->stream));
  CU(cudaMemsetAsync(c->stats, 0, sizeof(amm::DeviceStats), c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return AMM_OK;
}

}  // extern "C"
