// Internal definitions shared by the library's translation units: the
// context, the device data layout and the kernel launchers.
//
// Device layout (structure of arrays; "real" is double for the FP64 form and
// float for the FP32 forms; vectors are always 3-component, z = 0 in 2D):
//   per cell   Q      double, 5 planes of n: m, px, py, pz, E
//              cw     2 x R4<real>: {rho, vx, vy, vz}, {P, s - r}: one
//                     32-byte (FP32) record, so a gathered neighbour costs one sector
//              grad   4 x R4<real>: {d rho (xyz), dP/dx}, {d vx, dP/dy},
//                                   {d vy, dP/dz}, {d vz, 0}
//              cgeo   R4<real> {1/V, s - r}   crad real R_i   cgeo64 R4<double> {V, s - r}
//              wmesh  R4<real> {wx, wy, wz, 0} (explicit mesh velocity only)
//   per face   lr     int2 {L, R}
//              fgeo   2 x R4<real>: {n (unit, L->R), |r_R - r_L|}, {c = f - m, A}
//              flux   R4<real> {A F_m, A F_px, A F_py, A F_pz}, fluxE real A F_E
//   cell->face csr_off int [n+1], csr int2 {face << 1 | side, neighbour}
//              (side 0: the cell is the face's left cell), in face order.
//   per incidence (csr order; the gradient kernel streams them):
//              igAB 2 x R4<real>: {A (c / |d| + s n / 2), 0}, {f - s_i, j}
//                   (one 32-byte record in the FP32 forms; the neighbour j
//                   as the bits of the last real)
//              (s = +1 for the face's left cell, -1 for its right cell)
//   numbering  cells are renumbered along a Morton curve per box and faces
//              sorted by their new left cell; cell_perm / face_perm map back
//   tiles      contiguous cell / face ranges, each inside one box; one CTA
//              processes one tile, so per-box reductions never straddle boxes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "amm.h"

namespace amm {

template <typename real>
struct alignas(4 * sizeof(real)) R4 {
  real x, y, z, w;
};

constexpr int CELL_TILE = 256;   // cells per CTA
constexpr int FACE_TILE = 256;   // faces per CTA

struct Tile {
  int box;
  int begin;
  int end;
  int pad;
};

enum StatusBits : unsigned { ST_NEWTON_CAP = 1u, ST_NONPOS = 2u, ST_TIMEOUT = 4u, ST_DEPTH = 8u, ST_SUBSTEPS = 16u };

// per-box largest |A F| slots: m, p (3), E, and the entropy flux
constexpr int FMAX_STRIDE = 6;

struct DeviceStats {
  unsigned long long steps, faces, newton_iters, newton_fail, fallback, vacuum, guard, nonpos;
  unsigned int newton_max, status;
  unsigned long long hist[16];
  unsigned long long kept;
};

// The faces the plain FP32 flux kernel leaves to the learned proposal: a list
// of {face, box} of at most `capacity` entries and its length on the device.
struct FluxDefer {
  int2* list = nullptr;
  unsigned* count = nullptr;
  unsigned capacity = 0;
};

// Ideal-gas constants in the bulk arithmetic type, derived once on the host.
template <typename real>
struct GasC {
  real g, gm1, gp1;
  real z;            // (g-1)/(2g)
  real inv_z;        // 1/z
  real two_gm1;      // 2/(g-1)
  real gm1_gp1;      // (g-1)/(g+1)
  real two_gp1;      // 2/(g+1)
  real shock_a;      // (g+1)/(2g)
  real shock_b;      // (g-1)/(2g) = z
  real inv_g;        // 1/g
  real fan_rho;      // 2/(g-1)
  real fan_p;        // 2g/(g-1)
  real inv_gm1;      // 1/(g-1)
  GasC() = default;
  __host__ __device__ explicit GasC(double gamma) {
    g = (real)gamma;
    gm1 = (real)(gamma - 1.0);
    gp1 = (real)(gamma + 1.0);
    z = (real)((gamma - 1.0) / (2.0 * gamma));
    inv_z = (real)(2.0 * gamma / (gamma - 1.0));
    two_gm1 = (real)(2.0 / (gamma - 1.0));
    gm1_gp1 = (real)((gamma - 1.0) / (gamma + 1.0));
    two_gp1 = (real)(2.0 / (gamma + 1.0));
    shock_a = (real)((gamma + 1.0) / (2.0 * gamma));
    shock_b = (real)((gamma - 1.0) / (2.0 * gamma));
    inv_g = (real)(1.0 / gamma);
    fan_rho = (real)(2.0 / (gamma - 1.0));
    fan_p = (real)(2.0 * gamma / (gamma - 1.0));
    inv_gm1 = (real)(1.0 / (gamma - 1.0));
  }
};

// Kernel-side view of a context for one precision.
template <typename real>
struct HydroView {
  int dim, mode, limit, maxit, nboxes;
  int n, nf;
  int n_ctiles, n_ftiles;
  double gamma, tol;
  real tol_r;                  // tol in the bulk type
  GasC<real> gas;
  int fixed_acc;               // FP32 forms: exact int64 fixed-point flux sums
  int headroom;                // bits reserved for the incidence count in the fixed-point sums
  int update_lanes;            // lanes per cell of the update kernel (partial sums per block)
  unsigned* fmax_bits;         // [nboxes][FMAX_STRIDE] max |A F| per component (float bits) of the step
  // dt source: dt_box[b] if cfl <= 0, else cfl * courant_min[b]
  double cfl;
  const double* dt_box;
  double* dt_used;
  unsigned long long* cour_bits;
  double* Q;                  // 5 planes of n
  R4<real>* cw;                // [n][2] {rho, v}, {P, s - r}
  R4<real>* grad;
  // static mesh: each cell's state predicted over half the step in the lab
  // frame, W - (dt/2) A(W) grad W, written by the gradient kernel:
  // {rho, v}, {P, s - r} per cell, and A likewise with the entropy switch
  int pred;
  R4<real>* cwp;
  real* Apw;
  const R4<real>* wmesh;
  const R4<real>* cgeo;        // {1/V, s - r}
  const real* crad;            // effective radius R_i of eq. (EqnTiStep)
  const R4<double>* cgeo64;    // {V, s - r} in FP64
  const int2* lr;
  const R4<real>* fgeo;
  R4<real>* flux;
  real* fluxE;
  const int* csr_off;
  const int2* csr;
  const R4<real>* igAB;        // [2 q], [2 q + 1]
  const Tile* ctiles;
  const Tile* ftiles;
  const int* cell_perm;        // internal -> caller numbering
  const int* face_perm;
  double* partial;            // [n_ctiles][5]
  double* totals;             // [nboxes][5]
  const int* box_first_ctile; // [nboxes+1]
  DeviceStats* stats;
  unsigned* box_status;        // [nboxes] StatusBits of each box
  // mesh-regularity correction (Sec. 4.1)
  int regularize;
  real eta_r, chi_r;
  R4<real>* wcorr;             // [n] corrected generator velocities of the step
  // entropy switch (Sec. 3.5)
  int entropy;
  double mach_thresh, alpha_s;
  double* S;                   // [n] total entropy M A
  real* Aw;                    // [n] entropic function A = S / M of the current state
  R4<real>* gradA;             // [n] {limited grad A, 0}
  real* fluxS;                 // [nf] A F_S
  real* machf;                 // [nf] largest shock Mach number of the face's Riemann problem
  real* ekmax;                 // [n] largest kinetic energy of the cell and its neighbours
  unsigned char* kept;         // [n] 1 where the last update kept the advected entropy
  // learned proposal (FP32 learned form only)
  const void* mlp;
  float* harvest;              // if set, the flux kernel records each face's Riemann inputs [nf][6]
};

// Loop state of a cycle of individual time steps, in device memory: the
// cycle runs as a while loop inside one CUDA graph, and k_ind_next advances it.
struct IndLoop {
  long long tick;                   // current tick
  long long T;                      // ticks per cycle, 2^depth
  int stamp;                        // stamp of the current tick
  int deepest;                      // largest bin in use during the cycle
  int go;                           // 1 while the cycle continues
  int pad;
  unsigned long long substeps, face_fluxes, activations;
  unsigned long long max_substeps;  // the loop stops (ST_SUBSTEPS) beyond this
};

// Device state of the individual-step integrator (amm_ctx::ind).
struct IndView {
  int n, nf, dim, depth;            // depth: max_depth D (ticks per cycle 2^D)
  int levels;                       // pyramid levels 0..levels-1 (leaf = levels-1)
  int signal;                       // 1: signal-speed criterion, 0: eq. (EqnTiStep) alone
  double cfl, dtick, gamma;
  double box[3];
  const double* gen;                // [n][3] generators
  IndLoop* loop;                    // tick, stamp and counters
  cudaGraphConditionalHandle handle;  // the cycle's while condition
  int in_graph;                     // 1: k_ind_next sets the condition; 0: the host loops
  signed char* bin;                 // [n]
  unsigned char* act;               // [n] active at this tick
  int* list;                        // [n] active cells
  int* flist;                       // [nf] active faces
  int* count;                       // [0] active cells, [1] active faces
  int* fstamp;                      // [nf] stamp of the tick a face was last active
  int* cstamp;                      // [n]  stamp of the tick a cell was last touched
  double* fdt;                      // [nf] the active face's step
  unsigned* hist;                   // [64] cells per bin
  // pyramid: cells in leaf-bucket order
  const int* slot_cell;             // [n] slot -> cell
  const int* cell_slot;             // [n] cell -> slot
  const int* leaf_off;              // [leaf buckets + 1]
  DeviceStats* stats;               // status bits (the loop stops on a failure)
  double4* rec;                     // [n][2] by slot: {x, y, z, c}, {vx, vy, vz, |v|}
  float4* rec32;                    // the same in FP32 (the walk's first screen)
  float2* node;                     // per level, per bucket: {max (c + |v|) (-1: empty), its slot (int bits)}
  const int* level_off;             // [levels] first node of each level
};

}  // namespace amm

struct amm_ctx {
  int dim = 0;
  int64_t n = 0, nf = 0;
  int nboxes = 1;
  double gamma = 1.4;
  amm_options opt;
  cudaStream_t stream = nullptr;
  cudaStream_t aux_stream = nullptr;  // graph capture
  bool own_stream = false;
  std::string err;
  std::vector<int64_t> box_cells, box_faces;
  std::vector<double> box_h;       // [nboxes][3]
  int n_ctiles = 0, n_ftiles = 0;
  std::vector<int> box_first_ctile_h;
  // device memory
  double* gen = nullptr;           // [n][3]
  double* box = nullptr;           // [nboxes][3]
  double* Q = nullptr;             // [5][n]
  int2* lr = nullptr;
  int* csr_off = nullptr;
  int2* csr = nullptr;
  amm::Tile* ctiles = nullptr;
  amm::Tile* ftiles = nullptr;
  int* box_first_ctile = nullptr;
  int* cell_perm = nullptr;        // [n] internal cell -> caller's cell
  int* face_perm = nullptr;        // [nf] internal face -> caller's face
  std::vector<int> perm_h;         // host copy of cell_perm
  void* fgeo = nullptr;            // [nf][2] R4<real>
  void* igAB = nullptr;            // [2 nf][2] R4<real> per-incidence records
  void* cgeo = nullptr;            // [n] R4<real> {1/V, s - r}
  void* crad = nullptr;            // [n] real, effective radius
  amm::R4<double>* cgeo64 = nullptr;
  void* cw = nullptr;              // [n][2] R4<real> cell records
  void* grad = nullptr;
  void* cwp = nullptr;             // [n][2] R4<real>: half-step predicted records (static mesh)
  void* Apw = nullptr;             // [n] real: predicted entropic function (entropy switch)
  void* wmesh = nullptr;
  void* flux = nullptr;
  void* fluxE = nullptr;
  unsigned long long* cour_bits = nullptr;
  unsigned* fmax_bits = nullptr;   // [nboxes][FMAX_STRIDE]
  void* wcorr = nullptr;           // regularity correction: [n] R4<real>
  double* S = nullptr;             // entropy switch: [n] total entropy
  void* Aw = nullptr;              // [n] real
  void* gradA = nullptr;           // [n] R4<real>
  void* fluxS = nullptr;           // [nf] real
  void* machf = nullptr;           // [nf] real
  void* ekmax = nullptr;           // [n] real
  unsigned char* kept = nullptr;   // [n]
  int headroom = 7;
  int grad_lanes = 4;              // lanes per cell in the gradient kernel
  int update_lanes = 4;            // lanes per cell in the update kernel
  int flux_block = 256;            // threads (faces) per CTA of the flux kernel
  float tuned_ms = 0.f;
  int persistent = 0;              // 1: one cooperative launch per step (amm_advance)
  unsigned* barrier = nullptr;     // grid-barrier counter and generation
  double* dt_box = nullptr;
  double* dt_used = nullptr;
  double* partial = nullptr;
  double* totals = nullptr;
  amm::DeviceStats* stats = nullptr;
  unsigned* box_status = nullptr;  // [nboxes]
  float* closure = nullptr;        // [n] relative closure error (creation only)
  void* mlp = nullptr;             // device copy of the proposal weights (MlpDevice)
  int2* defer_list = nullptr;      // learned form: faces past the proposal's gate [nf_cap] {face, box}
  unsigned* defer_count = nullptr; // and their number
  float* harvest = nullptr;        // set only during amm_harvest
  bool mlp_loaded = false;
  double* scratch = nullptr;       // layout conversions for getters/setters
  void* geo_ws = nullptr;          // FP64 face geometry before the FP32 cast (grown on demand)
  size_t geo_ws_bytes = 0;
  void* tess_ws = nullptr;         // amm_retessellate: the GPU tessellation's workspace (amm::vor::TessWork)
  int64_t nf_cap = 0;              // faces the face-sized buffers hold
  size_t scratch_size = 0;         // in doubles
  unsigned long long* counter = nullptr;
  bool grads_fresh = false;
  bool totals_fresh = false;
  bool have_step = false;
  // captured step graph
  cudaGraphExec_t graph = nullptr;
  double graph_cfl = -1.0;
  bool graph_profiled = false;
  bool graph_persistent = false;
  // individual time steps (allocated by the first amm_advance_individual)
  bool ind_ready = false;
  int ind_levels = 0;
  int ind_stamp = 0;
  std::vector<int> ind_level_off_h;
  signed char* ind_bin = nullptr;
  unsigned char* ind_act = nullptr;
  int* ind_list = nullptr;
  int* ind_flist = nullptr;
  int* ind_count = nullptr;
  int* ind_fstamp = nullptr;
  int* ind_cstamp = nullptr;
  double* ind_fdt = nullptr;
  unsigned* ind_hist = nullptr;
  int* ind_slot_cell = nullptr;
  int* ind_cell_slot = nullptr;
  int* ind_leaf_off = nullptr;
  int* ind_level_off = nullptr;
  void* ind_rec = nullptr;         // double4 [n][2]
  void* ind_rec32 = nullptr;       // float4 [n][2]
  void* ind_node = nullptr;        // float2 per pyramid node
  amm::IndLoop* ind_loop = nullptr;
  cudaGraph_t ind_graph = nullptr;  // the cycle as one graph (while loop over ticks)
  cudaGraphExec_t ind_exec = nullptr;
  double ind_key[4] = {0, 0, 0, 0}; // cfl, dt_max, max_depth, signal of the captured graph
  bool ind_host_loop = false;       // ticks launched by the host (for profilers)
  // per-kernel timing: events recorded between the kernels of a step
  bool profiling = false;
  cudaEvent_t prof_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool is_fp64() const { return opt.precision == AMM_FP64; }
  size_t real_size() const { return is_fp64() ? 8 : 4; }
};

namespace amm {

// voronoi.cu: the GPU tessellation into a reusable workspace
namespace vor {
struct TessWork;
TessWork* work_new();
void work_free(TessWork* w);
// the last build's faces (device arrays owned by w): cells [F][2], shift [F][dim], area [F], centroid [F][dim]
void work_faces(const TessWork* w, const int32_t** cells, const int8_t** shift, const double** area,
                const double** cen);
int tess_build_work(TessWork* w, int dim, int64_t n, const double* gen_d, const double* box, cudaStream_t st,
                    bool check, int64_t* nf_out, int64_t* asym, double* max_rel);
const char* tess_last_error();
}  // namespace vor

// geometry.cu
cudaError_t launch_face_geometry(amm_ctx* c, const double* area, const double* cen, const int8_t* shift_d3);
cudaError_t launch_cell_geometry(amm_ctx* c);
cudaError_t launch_drift(amm_ctx* c, double dt);

// hydro_f64.cu / hydro_f32.cu
template <typename real>
HydroView<real> make_view(amm_ctx* c, double cfl);
template <typename real>
cudaError_t launch_primitives(amm_ctx* c);
// the Courant minimum (and the regularity-corrected mesh velocities) of the
// current state, then the gradients; cfl > 0: the step is cfl times the
// Courant minimum, else dt_box (the predicted records need it)
template <typename real>
cudaError_t launch_courant(amm_ctx* c);
template <typename real>
cudaError_t launch_gradients(amm_ctx* c, double cfl);
template <typename real>
cudaError_t launch_flux(amm_ctx* c, double cfl);
template <typename real>
cudaError_t launch_update(amm_ctx* c, double cfl);
template <typename real>
cudaError_t launch_finish(amm_ctx* c, double cfl);
template <typename real>
cudaError_t launch_set_state(amm_ctx* c, const double* Q_aos_device, unsigned long long* bad_count);
template <typename real>
cudaError_t launch_get_state(amm_ctx* c, double* Q_aos_device);
template <typename real>
cudaError_t launch_get_primitives(amm_ctx* c, double* W_aos_device);
template <typename real>
cudaError_t launch_get_gradients(amm_ctx* c, double* g_device);
template <typename real>
cudaError_t launch_get_flux(amm_ctx* c, double* F_device);
template <typename real>
cudaError_t launch_set_wmesh(amm_ctx* c, const double* w_aos_device);

// flux_learned.cu: the FP32 flux kernel with the fused proposal network, and
// the learned form's whole step as one cooperative launch
cudaError_t launch_flux_learned(amm_ctx* c, const HydroView<float>& v);
// flux_chunks.cu: the FP32 forms' flux kernel (learn: list the faces past the
// proposal's gate in `defer` instead of solving them)
cudaError_t launch_flux_chunks(amm_ctx* c, const HydroView<float>& v, bool learn, const FluxDefer& defer);
cudaError_t launch_step_persistent_learned(amm_ctx* c, double cfl);
cudaError_t prepare_flux_learned();

// hydro_f64.cu / hydro_f32.cu: one tick of individual time steps (Sec. 7.2)
template <typename real>
cudaError_t launch_individual_tick(amm_ctx* c, const IndView& d);
cudaError_t launch_individual_next(amm_ctx* c, const IndView& d);

// persistent_f32.cu / persistent_f64.cu: the whole step as one cooperative launch
template <typename real>
cudaError_t launch_step_persistent(amm_ctx* c, double cfl);

}  // namespace amm
