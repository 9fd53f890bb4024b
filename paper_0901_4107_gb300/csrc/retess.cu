// amm_retessellate: a new Voronoi mesh for a context's current generators,
// built on the GPU (amm_tess_build), with every cell keeping its conserved
// quantities -- the mesh step of the moving-mesh cycle (Sec. 3, step 8, then
// the next step's tessellation, Sec. 2) without leaving the device.
//
// The tessellation is built on the context's internal cell numbering, so the
// caller's numbering (cell_perm) is unchanged and the faces come out sorted by
// their left cell.  The cell -> face lists are rebuilt by a counting pass and
// ordered per cell as amm_create orders them (direction class of the outward
// normal, then larger faces first), so the result does not depend on the
// order in which the fill pass ran.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "amm_internal.cuh"

namespace amm {
namespace {

// the generators as [n][dim] (the context keeps them padded to 3)
__global__ void k_pack_gen(int n, int dim, const double* gen3, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < dim; d++) out[(size_t)i * dim + d] = gen3[(size_t)i * 3 + d];
}

// face inputs padded to 3 components: centroid and image shift
__global__ void k_pad_faces(int nf, int dim, const double* cen, const int8_t* shift, double* cen3, int8_t* sh3,
                            int* face_perm) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  for (int d = 0; d < 3; d++) {
    cen3[(size_t)k * 3 + d] = d < dim ? cen[(size_t)k * dim + d] : 0.0;
    sh3[(size_t)k * 3 + d] = d < dim ? shift[(size_t)k * dim + d] : 0;
  }
  face_perm[k] = k;
}

__global__ void k_csr_count(int nf, const int2* lr, int* count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int2 e = lr[k];
  atomicAdd(count + e.x, 1);
  atomicAdd(count + e.y, 1);
}

__global__ void k_scan_one(const int* count, int* start, int m) {
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

__global__ void k_csr_fill(int nf, const int2* lr, int* cursor, int2* csr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int2 e = lr[k];
  csr[atomicAdd(cursor + e.x, 1)] = make_int2(k << 1, e.y);
  csr[atomicAdd(cursor + e.y, 1)] = make_int2((k << 1) | 1, e.x);
}

// direction class of a vector: dominant axis and its sign, then the signs of
// the other components
__device__ __forceinline__ int klass(const double* d, int dim) {
  int ax = 0;
  for (int q = 1; q < dim; q++)
    if (fabs(d[q]) > fabs(d[ax])) ax = q;
  int cls = 2 * ax + (d[ax] < 0 ? 1 : 0);
  int sub = 0, bit = 0;
  for (int q = 0; q < dim; q++)
    if (q != ax) sub |= (d[q] < 0 ? 1 : 0) << (bit++);
  return cls * 4 + sub;
}

// each cell's list by (direction class of the outward normal, larger face
// first, face index); also the largest list length
__global__ void k_csr_sort(int n, int dim, const int* off, int2* csr, const int2* lr, const double* gen3,
                           const int8_t* sh3, const double* box3, const double* area, int* max_inc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lo = off[i], hi = off[i + 1];
  atomicMax(max_inc, hi - lo);
  auto key = [&](const int2& x, int& cls, double& a) {
    const int k = x.x >> 1;
    const int2 e = lr[k];
    double d[3];
    for (int q = 0; q < 3; q++)
      d[q] = gen3[(size_t)e.y * 3 + q] + sh3[(size_t)k * 3 + q] * box3[q] - gen3[(size_t)e.x * 3 + q];
    if (x.x & 1)
      for (int q = 0; q < 3; q++) d[q] = -d[q];
    cls = klass(d, dim);
    a = area[k];
  };
  for (int p = lo + 1; p < hi; p++) {
    const int2 v = csr[p];
    int cv;
    double av;
    key(v, cv, av);
    int q = p - 1;
    while (q >= lo) {
      int cq;
      double aq;
      key(csr[q], cq, aq);
      const bool after = cq > cv || (cq == cv && (aq < av || (aq == av && (csr[q].x >> 1) > (v.x >> 1))));
      if (!after) break;
      csr[q + 1] = csr[q];
      q--;
    }
    csr[q + 1] = v;
  }
}

}  // namespace
}  // namespace amm

extern "C" {

int amm_retessellate(amm_ctx* c) {
  using namespace amm;
  if (!c) return AMM_ERR_INVALID_ARG;
  if (c->nboxes != 1) {
    c->err = "amm_retessellate: one box only";
    return AMM_ERR_INVALID_ARG;
  }
  const int dim = c->dim;
  const int64_t n = c->n;
  cudaStream_t st = c->stream;
  std::string where;
  auto cu = [&](cudaError_t e, const char* w) {
    if (e != cudaSuccess && where.empty()) where = std::string(w) + ": " + cudaGetErrorString(e);
    return where.empty();
  };
  // 1. the tessellation of the current generators, internal numbering, into
  // the context's workspace (kept between calls)
  if (!c->tess_ws) c->tess_ws = vor::work_new();
  vor::TessWork* w = (vor::TessWork*)c->tess_ws;
  double* g = c->gen;
  if (dim != 3) {
    // [n][dim] in the workspace's volume scratch would be overwritten by the
    // build: a buffer of its own
    if (!cu(cudaMalloc(&g, sizeof(double) * n * dim), "alloc")) {
      c->err = where;
      return AMM_ERR_CUDA;
    }
    k_pack_gen<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int)n, dim, c->gen, g);
  }
  int64_t nf = 0;
  const int rc = vor::tess_build_work(w, dim, n, g, c->box_h.data(), st, false, &nf, nullptr, nullptr);
  if (dim != 3) cudaFree(g);
  if (rc != AMM_OK) {
    c->err = std::string("amm_retessellate: ") + vor::tess_last_error();
    return rc;
  }
  // 2. face-sized buffers: kept while the new face count fits, else grown
  // with room for the next meshes of the run
  const size_t rs = c->real_size();
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (c->ind_exec) cudaGraphExecDestroy(c->ind_exec);
  if (c->ind_graph) cudaGraphDestroy(c->ind_graph);
  c->ind_exec = nullptr;
  c->ind_graph = nullptr;
  if (nf > c->nf_cap) {
    const int64_t cap = nf + nf / 8;
    void** bufs[] = {(void**)&c->lr, (void**)&c->face_perm, (void**)&c->csr, &c->fgeo, &c->igAB, &c->flux, &c->fluxE, &c->fluxS, &c->machf, (void**)&c->ftiles,
                     (void**)&c->ind_flist, (void**)&c->ind_fstamp, (void**)&c->ind_fdt};
    const bool had_defer = c->defer_list != nullptr;
    if (had_defer) {
      cudaFree(c->defer_list);
      c->defer_list = nullptr;
    }
    for (void** b : bufs)
      if (*b) {
        cudaFree(*b);
        *b = nullptr;
      }
    cu(cudaMalloc(&c->lr, sizeof(int2) * cap), "alloc");
    cu(cudaMalloc(&c->face_perm, sizeof(int) * cap), "alloc");
    cu(cudaMalloc(&c->csr, sizeof(int2) * 2 * cap), "alloc");
    cu(cudaMalloc(&c->fgeo, rs * 8 * cap), "alloc");
    cu(cudaMalloc(&c->igAB, rs * 16 * cap), "alloc");
    cu(cudaMalloc(&c->flux, rs * 4 * cap), "alloc");
    cu(cudaMalloc(&c->fluxE, rs * cap), "alloc");
    if (c->opt.entropy) {
      cu(cudaMalloc(&c->fluxS, rs * cap), "alloc");
      cu(cudaMalloc(&c->machf, rs * cap), "alloc");
    }
    cu(cudaMalloc(&c->ftiles, sizeof(Tile) * ((cap + FACE_TILE - 1) / FACE_TILE)), "alloc");
    if (had_defer) cu(cudaMalloc((void**)&c->defer_list, sizeof(int2) * cap), "alloc");
    if (c->ind_ready) {
      cu(cudaMalloc(&c->ind_flist, sizeof(int) * cap), "alloc");
      cu(cudaMalloc(&c->ind_fstamp, sizeof(int) * cap), "alloc");
      cu(cudaMalloc(&c->ind_fdt, sizeof(double) * cap), "alloc");
      cu(cudaMemsetAsync(c->ind_fstamp, 0xff, sizeof(int) * cap, st), "memset");
    }
    if (where.empty()) c->nf_cap = cap;
  }
  if (nf != c->nf || c->n_ftiles == 0) {
    std::vector<Tile> ft;
    for (int64_t s = 0; s < nf; s += FACE_TILE) ft.push_back(Tile{0, (int)s, (int)std::min<int64_t>(s + FACE_TILE, nf), 0});
    c->n_ftiles = (int)ft.size();
    cu(cudaMemcpyAsync(c->ftiles, ft.data(), sizeof(Tile) * ft.size(), cudaMemcpyHostToDevice, st), "copy");
    cu(cudaStreamSynchronize(st), "sync");     // the host vector goes out of scope
    c->nf = nf;
    c->box_faces = {0, nf};
  }
  // 3. faces, cell -> face lists, geometry
  const int32_t* wcells;
  const int8_t* wshift;
  const double* warea;
  const double* wcen;
  vor::work_faces(w, &wcells, &wshift, &warea, &wcen);
  double* cen3 = nullptr;
  int8_t* sh3 = nullptr;
  int *count = nullptr, *cursor = nullptr, *maxinc = nullptr;
  const unsigned gf = (unsigned)((nf + 255) / 256), gc = (unsigned)((n + 255) / 256);
  if (where.empty() && cu(cudaMalloc(&cen3, sizeof(double) * 3 * nf), "alloc") &&
      cu(cudaMalloc(&sh3, 3 * nf), "alloc") && cu(cudaMalloc(&count, sizeof(int) * n), "alloc") &&
      cu(cudaMalloc(&cursor, sizeof(int) * n), "alloc") && cu(cudaMalloc(&maxinc, sizeof(int)), "alloc")) {
    cu(cudaMemcpyAsync(c->lr, wcells, sizeof(int2) * nf, cudaMemcpyDeviceToDevice, st), "copy");
    k_pad_faces<<<gf, 256, 0, st>>>((int)nf, dim, wcen, wshift, cen3, sh3, c->face_perm);
    cu(cudaMemsetAsync(count, 0, sizeof(int) * n, st), "memset");
    cu(cudaMemsetAsync(maxinc, 0, sizeof(int), st), "memset");
    k_csr_count<<<gf, 256, 0, st>>>((int)nf, c->lr, count);
    k_scan_one<<<1, 1024, 0, st>>>(count, c->csr_off, (int)n);
    cu(cudaMemcpyAsync(cursor, c->csr_off, sizeof(int) * n, cudaMemcpyDeviceToDevice, st), "copy");
    k_csr_fill<<<gf, 256, 0, st>>>((int)nf, c->lr, cursor, c->csr);
    k_csr_sort<<<gc, 256, 0, st>>>((int)n, dim, c->csr_off, c->csr, c->lr, c->gen, sh3, c->box, warea, maxinc);
    cu(cudaGetLastError(), "csr");
    int mi = 0;
    cu(cudaMemcpyAsync(&mi, maxinc, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
    cu(cudaStreamSynchronize(st), "sync");
    c->headroom = 1;
    while ((1 << c->headroom) < mi + 1) c->headroom++;
    c->headroom += 1;
    if (where.empty()) cu(launch_face_geometry(c, warea, cen3, sh3), "geometry");
    if (where.empty())
      cu(c->is_fp64() ? launch_primitives<double>(c) : launch_primitives<float>(c), "primitives");
    cu(cudaStreamSynchronize(st), "sync");
  }
  void* tmp[] = {cen3, sh3, count, cursor, maxinc};
  for (void* p : tmp)
    if (p) cudaFree(p);
  if (!where.empty()) {
    c->err = "amm_retessellate: " + where;
    return AMM_ERR_CUDA;
  }
  c->grads_fresh = false;
  c->totals_fresh = false;
  return AMM_OK;
}

// the current faces in the caller's cell numbering: cells [F][2], area [F]
int amm_get_faces(amm_ctx* c, int32_t* cells, double* area) {
  using namespace amm;
  if (!c || !cells || !area) return AMM_ERR_INVALID_ARG;
  std::vector<int2> lr((size_t)c->nf);
  const size_t rs = c->real_size();
  std::vector<unsigned char> fg(rs * 8 * (size_t)c->nf);
  if (cudaMemcpyAsync(lr.data(), c->lr, sizeof(int2) * c->nf, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(fg.data(), c->fgeo, fg.size(), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    c->err = "amm_get_faces: copy failed";
    return AMM_ERR_CUDA;
  }
  std::vector<int> fp((size_t)c->nf);
  if (cudaMemcpy(fp.data(), c->face_perm, sizeof(int) * c->nf, cudaMemcpyDeviceToHost) != cudaSuccess) return AMM_ERR_CUDA;
  for (int64_t k = 0; k < c->nf; k++) {
    const int64_t o = fp[k];
    cells[2 * o] = c->perm_h[lr[k].x];
    cells[2 * o + 1] = c->perm_h[lr[k].y];
    // {n, |d|}, {c, A}: A is the last component of the second record
    if (rs == 8)
      area[o] = reinterpret_cast<const R4<double>*>(fg.data())[2 * k + 1].w;
    else
      area[o] = reinterpret_cast<const R4<float>*>(fg.data())[2 * k + 1].w;
  }
  return AMM_OK;
}

int64_t amm_get_num_faces(const amm_ctx* c) { return c ? c->nf : 0; }

}  // extern "C"
