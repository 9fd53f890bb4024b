/*
 * amm.h -- C ABI of the GB300 moving-mesh hydro library (libamm.so).
 *
 * One second-order unsplit Godunov (MUSCL-Hancock) update of the ideal-gas
 * Euler equations on a given Voronoi tessellation, after Springel (2010),
 * "E pur si muove", Sec. 3: primitives, Voronoi gradients and slope limiter,
 * face velocities, the per-face flux in the frame of the moving face with an
 * exact Riemann solver, the conservative cell update, and the global Courant
 * time step (Sec. 7.1).  The tessellation is an input.
 *
 * Conventions shared by every call
 *  - Face k joins the left cell L = face_cells[2k] and the right cell
 *    R = face_cells[2k+1].  The right cell's generator is taken in its periodic
 *    image r_R + face_shift[k] * box (face_shift in box lengths, per axis), the
 *    face normal points from L to R, and face_centroid[k] is given in the left
 *    cell's frame.
 *  - Cell states are conserved totals Q_i = (m, p_1..p_dim, E) (Sec. 3, the
 *    integrals of rho, rho v and rho e over the cell), row-major [n][dim+2],
 *    FP64.  Primitives are W_i = (rho, v_1..v_dim, P).
 *  - Every pointer argument is a HOST pointer unless the name ends in _device.
 *    The library copies what it needs; the caller keeps ownership of all
 *    arrays it passes.
 *  - Every call returns an amm_status (0 = AMM_OK, negative = error).  Nothing
 *    aborts, traps or throws across the ABI.  amm_last_error() describes the
 *    most recent error of a context.
 *  - Work is queued on the context's CUDA stream and runs asynchronously;
 *    calls that return data to the host (amm_get_*, amm_timestep, amm_sync)
 *    synchronise that stream first.  Numeric problems found on the device
 *    (a Newton solve that hit its cap, a cell whose pressure or mass became
 *    non-positive) are reported as AMM_ERR_NUMERIC by the next synchronising
 *    call, with counts in amm_stats.
 *  - One context per stream; a context is not thread-safe.
 */
#ifndef AMM_H
#define AMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMM_OK = 0,
  AMM_ERR_INVALID_ARG = -1,        /* bad sizes, indices, pointers or options */
  AMM_ERR_OPEN_CELL = -2,          /* a cell is not closed: |sum_faces A n| > 1e-9 sum A, or V <= 0 */
  AMM_ERR_NONPOSITIVE_STATE = -3,  /* an input cell has m <= 0 or P <= 0 */
  AMM_ERR_CUDA = -4,               /* a CUDA runtime call failed (no device, out of memory, ...) */
  AMM_ERR_NUMERIC = -5,            /* device-side numeric failure; see amm_stats */
  AMM_ERR_NOT_READY = -6,          /* a prerequisite is missing (e.g. no proposal weights loaded) */
  AMM_ERR_TIMEOUT = -7             /* a bounded device-side wait ran out */
} amm_status;

typedef enum {
  AMM_FP64 = 0,          /* every step in FP64 */
  AMM_FP32 = 1,          /* FP32 bulk arithmetic; FP64 accumulation, Newton guard and sums */
  AMM_FP32_LEARNED = 2   /* AMM_FP32 with the learned p* proposal as the Newton start */
} amm_precision;

typedef enum {
  AMM_EULERIAN = 0,      /* w_i = 0: static mesh */
  AMM_LAGRANGIAN = 1,    /* w_i = v_i, eq. (eqnvelmesh) */
  AMM_EXPLICIT_W = 2     /* w_i given by amm_set_mesh_velocity */
} amm_mesh_motion;

typedef struct amm_options {
  int precision;            /* amm_precision */
  int mesh_motion;          /* amm_mesh_motion */
  int limiter;              /* 1: slope limiter of Sec. 3.1 on; 0: unlimited gradients */
  int max_iter;             /* Newton iteration cap (default 64); hitting it is AMM_ERR_NUMERIC */
  double riemann_tol;       /* relative Newton tolerance 2|dp|/(p_new+p_old); <= 0 picks
                               1e-12 for AMM_FP64 and 1e-6 for the FP32 forms */
  void* stream;             /* cudaStream_t to run on; NULL: the context creates its own */
  int64_t n_boxes;          /* independent periodic boxes in one context (ensemble), >= 1 */
  const int64_t* box_cells; /* [n_boxes+1] cell offsets of each box; NULL when n_boxes == 1 */
  const int64_t* box_faces; /* [n_boxes+1] face offsets of each box; NULL when n_boxes == 1 */
  int fp64_accumulate;      /* FP32 forms only.  0 (default): each cell sums its face fluxes exactly,
                               as int64 multiples of a per-box, per-component power of two, so the
                               update conserves exactly and is order independent; 1: sums in FP64
                               floating point (about 20x slower on GB300's FP64 pipe) */
  int entropy;              /* 1: entropy switch of Sec. 3.5.  The total entropy S = M A of each cell
                               (A = P / rho^gamma, reconstructed at the faces like the primitives) is
                               advected with the face fluxes rho_F u_F A_upwind; a cell keeps its
                               advected S and takes its thermal energy from it, P = (S/M) rho^gamma,
                               when the largest shock Mach number of its faces' Riemann problems is
                               below mach_thresh, or when alpha_s > 0 and its new thermal energy is
                               below alpha_s times the largest kinetic energy of the cell and its
                               neighbours (relative to the cell's mesh velocity, eq. eqnScrit1); other
                               cells keep the conservative energy update and re-initialise
                               S = M P / rho^gamma.  Total energy is then conserved only where no cell
                               kept its entropy.  0 (default): the plain energy update. */
  double mach_thresh;       /* shock Mach threshold of the switch (default 1.1) */
  double alpha_s;           /* cold-flow parameter (default 0.01; 0 disables that criterion) */
  int regularize;           /* 1: mesh-regularity correction of Sec. 4.1, eq. (EqnShapeCorrVel): a
                               generator further than eta R_i from its cell's centre of mass s_i gets
                               the extra velocity chi c_i (s_i - r_i)/|s_i - r_i| (ramped in between
                               0.9 and 1.1 eta R_i), in the face velocities, the Courant step and
                               amm_drift.  Moving meshes only (AMM_ERR_INVALID_ARG with AMM_EULERIAN).
                               0 (default): off. */
  double eta;               /* threshold fraction of the cell radius (default 0.25) */
  double chi;               /* strength, in units of the sound speed (default 1) */
} amm_options;

typedef struct amm_stats {
  int64_t steps;             /* updates applied since the last reset */
  int64_t faces;             /* face fluxes computed */
  int64_t newton_iters;      /* total Newton iterations */
  int64_t newton_fail;       /* faces whose Newton solve hit max_iter */
  int64_t fallback_faces;    /* faces whose extrapolated state was not positive (first order used) */
  int64_t vacuum_faces;      /* faces whose Riemann problem generated vacuum */
  int64_t guard_faces;       /* FP32 forms: faces whose Newton solve finished in FP64 */
  int64_t nonpositive_cells; /* cells left with m <= 0 or P <= 0 by an update */
  int32_t newton_max;        /* largest iteration count on one face */
  uint32_t status;           /* bit 0 Newton cap, bit 1 non-positive cell, bit 2 wait timeout,
                                bit 3 time bin deeper than max_depth, bit 4 more than 2^20 ticks in
                                one cycle (amm_advance_individual) */
  int64_t newton_hist[16];   /* faces by Newton iteration count 0..14, 15 and more */
  int64_t entropy_kept;      /* cell updates that kept the advected entropy (amm_options.entropy) */
} amm_stats;

typedef struct amm_ctx amm_ctx;

/* Fills *opt with the defaults: FP64, Lagrangian, limiter on, max_iter 64,
 * tolerance by precision, own stream, one box. */
void amm_default_options(amm_options* opt);

/* Creates a context for one tessellation (Sec. 3, step 1 done by the caller).
 *   dim            2 or 3
 *   n_cells        cells (= generators), all boxes together
 *   generators     [n_cells][dim] positions, inside [0, box) of their box
 *   n_faces        faces, all boxes together
 *   face_cells     [n_faces][2] left, right cell (global indices, same box)
 *   face_shift     [n_faces][dim] periodic image of the right cell, box lengths
 *   face_area      [n_faces] area (length in 2D), >= 0
 *   face_centroid  [n_faces][dim] centroid in the left cell's frame
 *   box            [n_boxes][dim] periodic box lengths
 *   cell_Q         [n_cells][dim+2] conserved totals
 *   gamma          adiabatic index, > 1
 *   opt            options; NULL for defaults
 * Derives on the device the cell volumes and centres of mass from the
 * pyramid sums of Sec. 2.3, the per-face geometry and the cell->face lists,
 * and validates the input.  Errors: AMM_ERR_INVALID_ARG, AMM_ERR_OPEN_CELL,
 * AMM_ERR_NONPOSITIVE_STATE, AMM_ERR_CUDA; *out is NULL on error. */
int amm_create(amm_ctx** out, int dim, int64_t n_cells, const double* generators, int64_t n_faces,
               const int32_t* face_cells, const int8_t* face_shift, const double* face_area,
               const double* face_centroid, const double* box, const double* cell_Q, double gamma,
               const amm_options* opt);

/* The same from device arrays: generators, face_cells, face_shift, face_area,
 * face_centroid and cell_Q are device pointers (layouts as above), box (and
 * the options' box offsets) stay on the host.  The arrays are borrowed for
 * the call only: they are copied (through host memory, where the face list is
 * ordered and checked), so the caller keeps ownership.  Errors as amm_create,
 * plus AMM_ERR_CUDA if a copy fails.  Synchronises. */
int amm_create_device(amm_ctx** out, int dim, int64_t n_cells, const double* generators_device, int64_t n_faces,
                      const int32_t* face_cells_device, const int8_t* face_shift_device,
                      const double* face_area_device, const double* face_centroid_device, const double* box,
                      const double* cell_Q_device, double gamma, const amm_options* opt);

/* Releases all device memory of the context.  NULL is accepted. */
int amm_destroy(amm_ctx* ctx);

/* Message of the last error on this context (never NULL). */
const char* amm_last_error(const amm_ctx* ctx);

/* Replaces the cell states; host [n_cells][dim+2] or device (same layout).
 * Checks m > 0 and P > 0 (AMM_ERR_NONPOSITIVE_STATE).  Used for
 * checkpoint/resume: a resumed run is bitwise identical to an uninterrupted one.
 * With the entropy switch, also sets each cell's entropy to S = M P / rho^gamma
 * (a resumed run then also needs amm_set_entropy). */
int amm_set_state(amm_ctx* ctx, const double* Q);
int amm_set_state_device(amm_ctx* ctx, const double* Q_device);

/* Entropy switch (amm_options.entropy): the cells' total entropies S = M A,
 * host [n_cells]; amm_get_entropy also returns, if kept != NULL, 1 for the
 * cells that kept their advected entropy in the last step, else 0 ([n_cells]).
 * AMM_ERR_INVALID_ARG on a context without the switch, or for S <= 0. */
int amm_get_entropy(amm_ctx* ctx, double* S, uint8_t* kept);
int amm_set_entropy(amm_ctx* ctx, const double* S);

/* Mesh-generator velocities for AMM_EXPLICIT_W, host [n_cells][dim] (Sec. 3.2). */
int amm_set_mesh_velocity(amm_ctx* ctx, const double* w);

/* Sec. 3, step 3: primitives, Voronoi gradients (eq. eqngrad2) and the slope
 * limiter for the current state; also the per-box Courant minimum used by
 * amm_timestep.  Queued on the stream. */
int amm_gradients(amm_ctx* ctx);

/* Sec. 7.1, eq. (EqnTiStep): dt_out[b] = cfl * min_i R_i / (c_i + |v_i - w_i|)
 * over the cells of box b; host array of n_boxes.  One pass over the current
 * state's cells (with the mesh-regularity correction it also sets the
 * corrected mesh velocities that amm_drift takes).  Synchronises. */
int amm_timestep(amm_ctx* ctx, double cfl, double* dt_out);

/* Sec. 3, steps 3-7: gradients and limiter of the current state (on a static
 * mesh also each cell's state predicted over dt/2, which this dt sets), face
 * velocities, fluxes, conservative update with time step dt (every box), then
 * the primitives of the new state and the conservation sums. */
int amm_step(amm_ctx* ctx, double dt);
/* Same with one time step per box, host [n_boxes]. */
int amm_step_boxes(amm_ctx* ctx, const double* dt);

/* nsteps complete steps (gradients, Courant step with coefficient cfl per box,
 * fluxes, update), the time step staying on the device; replayed from a
 * captured CUDA graph when use_graph != 0.  Does not synchronise. */
int amm_advance(amm_ctx* ctx, double cfl, int64_t nsteps, int use_graph);

/* ---------------------------------------------------------------------------
 * Voronoi tessellation on the GPU (Sec. 2): the face list consumed by
 * amm_create / amm_create_device, built from device-resident generators.
 * Each cell is the intersection of the half-spaces bounded by the bisectors to
 * nearby generators and their periodic images; candidates are searched in
 * shells of a uniform grid until the completeness radius is reached (twice
 * the largest vertex distance, Sec. 2.4).  Faces of zero area (below 1e-12
 * h^(dim-1), h the mean spacing) are dropped.  A face is listed once, by the
 * cell with the smaller index (by the side with a positive image shift for a
 * face with its own image), with the right cell's periodic image in box
 * lengths and the centroid in the left cell's frame -- the layout amm_create
 * takes.  3D: one warp per cell, at most 64 faces per cell; 2D: 32.
 * --------------------------------------------------------------------------- */
typedef struct amm_tess amm_tess;

/* gen_device: [n][dim] device array, every coordinate in [0, box[d]);
 * box: host [dim]; stream: cudaStream_t or NULL.  Synchronises.  Errors:
 * AMM_ERR_INVALID_ARG (bad sizes, a generator outside the box),
 * AMM_ERR_NUMERIC (a cell over capacity, vanished -- duplicate generators --,
 * not closed, or incomplete; amm_tess_last_error says which), AMM_ERR_CUDA. */
int amm_tess_build(amm_tess** out, int dim, int64_t n, const double* gen_device, const double* box, void* stream);
const char* amm_tess_last_error(void);
int64_t amm_tess_num_faces(const amm_tess* t);
/* Device arrays owned by t: cells [F][2] (left, right), shift [F][dim],
 * area [F], centroid [F][dim] (absolute, left cell's frame). */
int amm_tess_faces(const amm_tess* t, const int32_t** cells, const int8_t** shift, const double** area,
                   const double** centroid);
/* Device arrays owned by t: cell volume [n] and centre of mass [n][dim]
 * (absolute), integrated from the cell's faces as pyramids about its
 * generator; half-faces per cell [n] (before the listing rule). */
int amm_tess_cells(const amm_tess* t, const double** volume, const double** com, const int32_t** faces_per_cell);
/* Listed faces whose mirror the neighbour did not find, and the largest
 * relative area mismatch between the two sides of a face. */
int amm_tess_check(const amm_tess* t, int64_t* asymmetric, double* max_rel);
int amm_tess_destroy(amm_tess* t);

/* The mesh step of the moving-mesh cycle on the device: a new Voronoi
 * tessellation of the context's current generators (after amm_drift) built on
 * the GPU as amm_tess_build does, replacing the context's faces; every cell
 * keeps its conserved quantities (and entropy), its primitives are recomputed
 * with its new volume.  One box only (AMM_ERR_INVALID_ARG otherwise).  The
 * face count usually changes: amm_get_num_faces and amm_get_faces give the
 * new list (face getters follow it).  Synchronises.  Errors as
 * amm_tess_build. */
int amm_retessellate(amm_ctx* ctx);
int64_t amm_get_num_faces(const amm_ctx* ctx);
/* The current faces in the caller's cell numbering: cells [F][2] (left,
 * right), area [F], host arrays. */
int amm_get_faces(amm_ctx* ctx, int32_t* cells, double* area);

/* Counters of one cycle of individual time steps. */
typedef struct amm_cycle_stats {
  int64_t substeps;     /* ticks at which steps started */
  int64_t face_fluxes;  /* face flux evaluations (a global step costs n_faces) */
  int64_t activations;  /* cell steps begun */
  int32_t deepest_bin;  /* largest bin in use during the cycle */
  int32_t reserved;
} amm_cycle_stats;

/* Sec. 7.2: one cycle of individual power-of-two time steps of total length
 * dt_max, on the static mesh (AMM_EULERIAN, one box, entropy switch off;
 * otherwise AMM_ERR_INVALID_ARG).  Cell i steps by dt_max / 2^b_i, the largest
 * such step not above its criterion dt_i = cfl min(tau_i, R_i/(c_i + |v_i|))
 * of eq. (EqnTiStepIndividual) (signal_speed != 0; tau_i, the shortest
 * signal travel time to any other cell, through the nearest periodic image,
 * is found by a pruned walk over a uniform-grid pyramid of the box) or of
 * eq. (EqnTiStep) alone (signal_speed == 0).  Time runs in ticks of
 * dt_max / 2^max_depth (1 <= max_depth <= 40); at each tick where steps
 * start, the starting cells take new primitives, limited gradients (the
 * other cells enter with the primitives of their own last start) and bins (a
 * shorter step is always allowed, a longer one is at most twice the current
 * step and only where that step also starts at this tick); every face with a starting cell is integrated over the shorter
 * step of its two cells, each side predicted from its own last start to the
 * middle of that step, and both cells exchange dt_f A F.  Every cell ends the
 * cycle synchronised, with fresh primitives.  The cycle runs on the device
 * as one CUDA graph (a while loop over the ticks; captured again when cfl,
 * dt_max, max_depth or signal_speed change) and synchronises once, at its
 * end.  stats may be NULL.  AMM_ERR_NUMERIC if a criterion fell below
 * dt_max / 2^max_depth (status bit 3), the cycle needed more than 2^20 ticks
 * (bit 4) or a Newton solve or cell failed; the loop stops at the first
 * failing tick. */
int amm_advance_individual(amm_ctx* ctx, double cfl, double dt_max, int max_depth, int signal_speed,
                           amm_cycle_stats* stats);

/* enable != 0: amm_advance_individual launches each tick from the host and
 * synchronises once per tick instead of running the cycle as one graph (the
 * same kernels and results; for profilers that cannot look inside graphs
 * with conditional nodes).  Default 0. */
int amm_individual_host_loop(amm_ctx* ctx, int enable);

/* The bins b_i in use at the end of the last cycle (step dt_max / 2^b_i),
 * host [n_cells]. */
int amm_get_bins(amm_ctx* ctx, int32_t* bins);

/* A10 (Sec. 3, step 8): moves the stored generators by w_i * dt (wrapped into
 * the box) for the caller's next tessellation. */
int amm_drift(amm_ctx* ctx, double dt);

/* Waits for queued work; returns AMM_ERR_NUMERIC if the device flagged a
 * numeric failure since the last reset, AMM_ERR_TIMEOUT for a timed-out wait. */
int amm_sync(amm_ctx* ctx);

/* Getters (synchronise).  Host arrays sized as documented. */
int amm_get_state(amm_ctx* ctx, double* Q);                 /* [n_cells][dim+2] */
int amm_get_state_device(amm_ctx* ctx, double* Q_device);   /* [n_cells][dim+2], device */
int amm_get_primitives(amm_ctx* ctx, double* W);            /* [n_cells][dim+2] */
int amm_get_gradients(amm_ctx* ctx, double* grad);          /* [n_cells][dim+2][dim], limited */
int amm_get_face_flux(amm_ctx* ctx, double* AF);            /* [n_faces][dim+2], area times flux of the last step */
int amm_get_geometry(amm_ctx* ctx, double* V, double* s);   /* [n_cells], [n_cells][dim] (s absolute) */
int amm_get_totals(amm_ctx* ctx, double* tot);              /* [n_boxes][dim+2], FP64 sums after the last step */
int amm_get_dt(amm_ctx* ctx, double* dt);                   /* [n_boxes], time step of the last step */
int amm_get_generators(amm_ctx* ctx, double* gen);          /* [n_cells][dim] */
int amm_get_stats(amm_ctx* ctx, amm_stats* stats);
/* Per-box status bits since the last reset, host [n_boxes] (bit 0 Newton cap,
 * bit 1 non-positive cell): boxes are independent, so a failed box does not
 * affect the others, which complete normally. */
int amm_get_box_status(amm_ctx* ctx, uint32_t* status);
int amm_reset_stats(amm_ctx* ctx);

/* Per-kernel timing for roofline measurements.  With profiling on, every
 * step records CUDA events on the context's stream between its kernels (also
 * inside a captured step graph, as external event nodes);
 * amm_get_kernel_times waits for the last step and returns the durations in
 * ms of its four kernel groups: [0] gradients+limiter+Courant, [1] face
 * fluxes, [2] cell update, [3] totals.  AMM_ERR_NOT_READY when profiling is
 * off.  Switching profiling re-captures the step graph. */
int amm_profile(amm_ctx* ctx, int enable);
int amm_get_kernel_times(amm_ctx* ctx, float* ms);

/* Launch shapes.  grad_lanes / update_lanes: consecutive threads that share
 * one cell in the gradient and update kernels (1, 2, 4 or 8); flux_block:
 * faces (threads) per CTA of the flux kernel (128 or 256).  Results do not
 * depend on them except for the FP64 rounding order of sums. */
typedef struct amm_tuning {
  int grad_lanes;
  int update_lanes;
  int flux_block;
  int persistent;  /* 1: amm_advance runs each step as ONE cooperative launch whose CTAs walk
                      every phase (gradients, fluxes, update, totals) with grid barriers between
                      them (bounded waits); 0: one launch per phase.  Both modes give
                      bit-identical states in the FP64 and FP32 forms; in the learned form
                      they agree to FP32 rounding (two kernels, two register budgets). */
  float step_ms;   /* amm_autotune: sum of the chosen kernels' median times */
} amm_tuning;

int amm_set_tuning(amm_ctx* ctx, const amm_tuning* t);
int amm_get_tuning(amm_ctx* ctx, amm_tuning* t);

/* Times every launch shape on this context's own mesh and state (reps steps
 * each from the same state, restored afterwards; device events on the
 * context's stream), keeps the fastest per kernel, then times whole steps
 * of that kernel sequence against the persistent single launch and keeps
 * the faster; returns the choice in *out (may be NULL).  Synchronises;
 * allocates one state-sized temporary. */
int amm_autotune(amm_ctx* ctx, double cfl, int reps, amm_tuning* out);

/* ---------------------------------------------------------------------------
 * Learned starting value for the Riemann star pressure (FP32 learned form).
 * The paper has no such component: a 6 -> 64 -> 64 -> 1 perceptron with SiLU
 * activations maps the normalised face state
 *   x = (log(rho_L/rhobar), log(p_L/pbar), u_L/cbar, log(rho_R/rhobar), log(p_R/pbar), u_R/cbar)
 * (rhobar, pbar the two-sided means, cbar = sqrt(gamma pbar/rhobar)) to
 * y = log(pstar / pbar); Newton then starts from pbar exp(y) and still runs to the
 * same tolerance.  Weights are BF16 on BF16 tensor cores with FP32
 * accumulation; FP32 master parameters are kept for training.
 * Parameter vector (AMM_MLP_NPARAMS floats): W1[64][6], b1[64], W2[64][64],
 * b2[64], W3[64], b3 (row = output unit).
 * Face states are [n][6] floats (rho_L, u_L, p_L, rho_R, u_R, p_R), u along
 * the face normal in the face frame.  *_device pointers are device memory;
 * calls on a handle run on its stream and the ones returning data to the
 * host synchronise it. */
#define AMM_MLP_NPARAMS 4673
typedef struct amm_mlp amm_mlp;
int amm_mlp_create(amm_mlp** out, double gamma, void* stream);
void amm_mlp_destroy(amm_mlp* net);
const char* amm_mlp_last_error(const amm_mlp* net);
int amm_mlp_num_params(void);
int amm_mlp_set_params(amm_mlp* net, const float* params);          /* host [AMM_MLP_NPARAMS] */
int amm_mlp_get_params(amm_mlp* net, float* params);                /* host [AMM_MLP_NPARAMS] */
/* y_device[i] = network(x_device[i]) for n feature rows [n][6] (tensor cores) */
int amm_mlp_forward(amm_mlp* net, const float* x_device, int64_t n, float* y_device);
/* Loss L = sum_i (y_i - t_i)^2 / n over the samples idx_device[0..n) (or
 * 0..n when idx_device is NULL) of x_device [.][6] and targets t_device, and
 * its gradient (host [AMM_MLP_NPARAMS], same order as the parameters) from
 * the tensor-core forward and backward passes.  Synchronises. */
int amm_mlp_grads(amm_mlp* net, const float* x_device, const float* t_device, const int32_t* idx_device, int64_t n,
                  float* grads, float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * FP32 master parameters with the gradient of that minibatch; the BF16
 * weights are refreshed.  Asynchronous; loss_device (may be NULL) receives
 * the minibatch loss.  amm_mlp_sync waits and reports a timed-out wait. */
int amm_mlp_train_step(amm_mlp* net, const float* x_device, const float* t_device, const int32_t* idx_device,
                       int64_t n, float lr, float* loss_device);
int amm_mlp_sync(amm_mlp* net);
/* Copies the network's BF16 weights into a context of the FP32 learned form
 * (AMM_FP32_LEARNED); its steps then start every Newton solve from the
 * network's proposal.  Steps of that form fail with AMM_ERR_NOT_READY before. */
int amm_mlp_attach(amm_ctx* ctx, const amm_mlp* net);
/* One step with device-side Courant time step (coefficient cfl), recording
 * every face's Riemann inputs after extrapolation, prediction and rotation
 * into states_device [n_faces][6] (internal face order) -- training data for
 * the proposal network.  FP32 forms only. */
int amm_harvest(amm_ctx* ctx, double cfl, float* states_device);
/* From face states [n][6] (rho_L, u_L, p_L, rho_R, u_R, p_R): the network's
 * features [n][6], and (each may be NULL) pbar [n], the two-shock estimate
 * p_TS [n] that the proposal corrects (p0 = p_TS exp(y)), and the compression
 * ratio ppv / max(p_L, p_R) [n] of the gate (the proposal is used where it
 * exceeds AMM_PROPOSAL_GATE); FP32, as the flux kernel computes them. */
#define AMM_PROPOSAL_GATE 1.25
int amm_mlp_features(double gamma, int64_t n, const float* states_device, float* x_device, float* pbar_device,
                     float* pts_device, float* ratio_device, void* stream);
/* the training target of each face state [n]: log(p* / p_TS), with p* the
 * exact star pressure (FP64 Newton from the standard guess to the relative
 * tolerance tol) and p_TS the two-shock estimate in FP32 as the flux kernel
 * forms it; NaN where the states generate vacuum or Newton did not converge */
int amm_mlp_targets(double gamma, int64_t n, const float* states_device, double tol, float* target_device,
                    void* stream);
/* exact star pressure of each face state in FP64 (Newton from the standard
 * guess to the relative tolerance tol); NaN where the states generate vacuum */
int amm_riemann_pstar(double gamma, int64_t n, const float* states_device, double tol, float* pstar_device,
                      void* stream);

/* Throughput probe of the arithmetic pipes (the paper has no counterpart: it
 * is the denominator of the ALU rooflines reported for the Riemann kernels).
 * Runs independent fused multiply-add chains, FP32 (fp64 = 0) or FP64
 * (fp64 = 1), on every SM of the current device: `iters` iterations of 8
 * chains per thread, 4 CTAs of 256 threads per SM.  Blocks until done.
 *   flop_out  host, receives the FLOPs performed (2 per FMA)
 *   ms_out    host, receives the kernel's device time (CUDA events)
 *   stream    cudaStream_t (NULL: the legacy default stream)
 * Errors: AMM_ERR_INVALID_ARG (iters < 1, NULL outputs), AMM_ERR_CUDA. */
int amm_alu_peak(int fp64, int iters, double* flop_out, float* ms_out, void* stream);

/* Allocation-free Courant time step.  The paper has no counterpart to this
 * entry point: it exists for callers that cannot allocate device memory --
 * code whose device memory is owned by another allocator (for example a
 * framework's caching pool that has reserved most of HBM) or that must not
 * call cudaMalloc/cudaFree on a latency-critical path, since those calls can
 * synchronise the device.  It computes the same quantity as amm_timestep for
 * one box, dt = cfl * min_i R_i / (c_i + |v_i - w_i|), from caller-owned
 * device arrays, without a context:
 *   W_device      [n_cells][dim+2] primitives (rho, v, P), FP64, device
 *   V_device      [n_cells] cell volumes, FP64, device
 *   wmesh_device  [n_cells][dim] mesh velocities, or NULL for a static mesh
 *   dt_device     one FP64 on the device, receives dt
 *   stream        cudaStream_t (NULL: the legacy default stream)
 * The call is asynchronous on `stream`.  Its only working memory is a static
 * device array of AMM_NOALLOC_MAX_BLOCKS doubles (128 KiB) that every GPU
 * loading the library holds until exit; hence at most AMM_NOALLOC_MAX_CELLS
 * cells (AMM_ERR_INVALID_ARG beyond).  The first call on each device looks up
 * the array's device address (with that device current) and should come
 * before any stream capture.  All calls share the array, so calls whose
 * kernels overlap on the GPU race; order them on one stream.
 * Errors: AMM_ERR_INVALID_ARG, AMM_ERR_CUDA. */
#define AMM_NOALLOC_MAX_BLOCKS 16384
#define AMM_NOALLOC_MAX_CELLS ((int64_t)AMM_NOALLOC_MAX_BLOCKS * 4096)
int amm_timestep_noalloc(int dim, int64_t n_cells, const double* W_device, const double* V_device,
                         const double* wmesh_device, double gamma, double cfl, double* dt_device, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AMM_H */
