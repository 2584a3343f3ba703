/*
 * bgk.h -- C ABI of the B300 implicit sweep solver for the multidimensional BGK equation
 * (Hauck et al., "Sweep-based, implicit solutions of the multidimensional BGK equation on
 * unstructured grids").
 *
 * Conventions shared by every call
 *   - Every call returns an int status (BGK_OK = 0 or one of BGK_E_*).  No exception or
 *     signal crosses the ABI; outputs are written only when the call returns BGK_OK.
 *   - Pointers named h_* are host memory; pointers named d_* are device memory on the
 *     handle's device.  Inputs are copied; the caller keeps ownership of every buffer.
 *   - The handle owns all device memory it allocates; it is not thread-safe.
 *   - Spatial DG nodes of a cell are ordered: P1 triangle/tetrahedron = its vertices in the
 *     order given; P2 triangle = vertices 0,1,2 then midpoints of edges (0,1),(1,2),(2,0).
 *     A "node index" is cell * n_dof + local node.  n_nodes = n_cells * n_dof.
 *   - Ordinates: velocity points v_j of the tensor grid on [-L, L]^d, j lexicographic with
 *     the last dimension fastest.  Distribution arrays are f[j][node] (ordinate-major).
 *   - Nodal states are [node][d+2] = (n, u_1..u_d, theta); moments are [node][d+2] =
 *     (n, n u_1..n u_d, E) with E = |u|^2 n / 2 + d n theta / 2   (Sec. 2, Eq. moments).
 */
#ifndef BGK_B300_H
#define BGK_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BGK_OK = 0,
  BGK_E_INVALID = 1,      /* bad argument or mesh (non-conforming, degenerate cell, ...) */
  BGK_E_CUDA = 2,         /* a CUDA runtime call failed */
  BGK_E_OOM = 3,          /* device allocation failed */
  BGK_E_NOCONV = 4,       /* Picard iteration reached l_max without meeting the criterion */
  BGK_E_NONPHYSICAL = 5,  /* n <= 0, theta <= 0 or a non-finite moment was met */
  BGK_E_TIMEOUT = 6,      /* a bounded device-side wait ran out */
  BGK_E_IO = 7            /* a checkpoint file could not be written or read, or does not match */
};

enum { BGK_BE = 0, BGK_DIRK2 = 1, BGK_DIRK3 = 2, BGK_BSTABLE2 = 3, BGK_BDF2 = 4 };
enum { BGK_COLL_MAXWELLIAN = 0, BGK_COLL_LINEAR = 1, BGK_COLL_INTERP = 2 };
/* Boundary conditions of Sec. 4.2 on the sides of a box domain.  INFLOW: given data g
 * (bgk_set_inflow_maxwellian / bgk_set_inflow).  BOUNCE_BACK: f^bc(x, v) = f(x, -v).
 * REFLECT: f^bc(x, v) = f(x, R_n v), R_n v = v - 2 (v.n) n (specular). */
enum { BGK_BC_INFLOW = 0, BGK_BC_BOUNCE_BACK = 1, BGK_BC_REFLECT = 2 };
/* BGK_FP64: FP64 storage and sweeps.  BGK_FP32_SWEEP: FP32 storage and sweeps, moments
 * and Maxwellian parameters to FP64 accuracy; it stalls at FP32 rounding (~1e-7 in the
 * moment change).  BGK_MIXED: FP64 state; each stage first runs FP32 sweeps until the
 * measure falls below max(tau', fp32_floor), then FP64 sweeps to tau' -- the converged
 * state is the FP64 one. */
enum { BGK_FP64 = 0, BGK_FP32_SWEEP = 1, BGK_MIXED = 2 };
enum { BGK_DTYPE_F64 = 0, BGK_DTYPE_F32 = 1 };

/* Mesh of the spatial domain X (Sec. 3.1, Table 1): affine simplices, conforming. */
typedef struct {
  int dim;                      /* 2 (triangles or quadrilaterals) or 3 (tetrahedra) */
  int k_x;                      /* spatial degree: 1, or 2 for triangles */
  int n_vertices;
  const double* xyz;            /* host, [n_vertices][dim] */
  int n_cells;
  const int32_t* cell_vertices; /* host, [n_cells][dim+1] (simplices, either orientation) or
                                   [n_cells][4] (quadrilaterals: vertices in order around the
                                   cell, either direction) */
  int shape;                    /* 0: simplices; 1: Q1 quadrilaterals (dim 2, k_x 1; Sec. 3.1's
                                   bilinear element), which must be parallelograms (x0 + x2 =
                                   x1 + x3 to 1e-12 of the cell size), else BGK_E_INVALID */
} bgk_mesh;

/* Velocity grid (Sec. 3.2): n_points per dimension on [-L, L], k_v+1 Gauss-Legendre
 * points in each of n_points/(k_v+1) uniform cells; nodal Q^{k_v} basis.  n_points <= 128
 * (BGK_E_INVALID above). */
typedef struct {
  double L;
  int n_points;
  int k_v;
} bgk_vgrid;

/* Physics and time integration (Sec. 2, Sec. 3.5, App. A, Sec. 5). */
typedef struct {
  double nu;          /* collision frequency (= 1/Knudsen) */
  int integrator;     /* BGK_BE, BGK_DIRK2, BGK_DIRK3, BGK_BSTABLE2, BGK_BDF2 */
  double dt;          /* time step; if <= 0, dt = cfl * dt_e (explicit bound of Sec. 5) */
  double cfl;
  int collision;      /* BGK_COLL_MAXWELLIAN (0): nu (M[f] - f) with the projected Maxwellian
                         (App. B); BGK_COLL_LINEAR (1): the simplified, linear Maxwellian
                         N_h = n / |V| at every ordinate, |V| = (2L)^d (Eq. linear-Maxwellian,
                         Prop. Linear Stability); it conserves mass only; BGK_COLL_INTERP (2):
                         the Maxwellian of the current moments evaluated at the grid points
                         (interpolation in velocity, the alternative Sec. 5.1.1 compares the
                         projection with); it does not conserve the moments exactly */
  int walls[6];       /* boundary condition per side of the box, BGK_BC_*, in the order
                         x-, x+, y-, y+, z-, z+ (the first 2d are read).  A boundary face
                         belongs to side (a, +/-) when its unit outward normal is +/-e_a
                         (other components below 1e-10 of its length); faces with any
                         other normal stay INFLOW.  BOUNCE_BACK and REFLECT couple ordinate
                         j to its mirror (-v_j, or v_j with component a negated; both are
                         grid points of the symmetric velocity grid) and read the mirror's
                         trace from the previous Picard iterate f^l (lagged, Sec. 4.2), so
                         the wall data are refreshed before every sweep.  All zero: inflow
                         everywhere. */
} bgk_physics;

/* Solver configuration. */
typedef struct {
  double tau;         /* Picard tolerance of Eq. (convergence-criteria); default 1e-8 */
  int l_max;          /* Picard iteration limit; default 1000 */
  int precision;      /* BGK_FP64 or BGK_FP32_SWEEP (FP32 sweep, FP64 moments) */
  int block_threads;  /* sweep CTA size override (0 = default) */
  void* stream;       /* cudaStream_t to run on (NULL = a stream owned by the handle) */
  int eager;          /* 0: each step is one CUDA graph (conditional while-node per stage);
                         1: the same kernels launched from a host loop (profiling aid) */
  int cache_inverse;  /* local-inverse cache for the stage coefficient: 0 = FP64 sweeps when it fits
                         in half of the free device memory, 1 = always (BGK_E_OOM if it cannot),
                         2 = never (assemble and factorise every local matrix in the sweep) */
  double fp32_floor;  /* BGK_MIXED: the FP32 phase stops below this measure (0 = 2e-7) */
  int prefetch;       /* sweep with cached inverses: 1 = copy each thread's next local inverse and
                         geometry to shared memory ahead of use (cp.async); otherwise read in
                         place (FP32 sweeps carry the next cell's geometry in registers) */
  int sweep_mode;     /* sweep algorithm (Sec. 4.1): 0 or 1 = TGS (a CTA per ordinate walks
                         the generations, the cells of a generation in parallel: the default),
                         2 = TS (a thread per ordinate walks its whole schedule alone).  Both
                         give the same results up to rounding.  TS wins only on narrow
                         domains with many ordinates (the Sod strip from 96x96 velocities);
                         bgk_autotune_sweep chooses by measurement */
  int sweep_front;    /* FP32 and float-pair generation sweeps of 2D meshes: 0 = read the
                         upwind traces that the sweep itself produced from a shared-memory
                         buffer when every ordinate's live front fits (slots assigned once at
                         creation; float-pair sweeps of at most 64 threads per CTA), else from
                         global memory; 2 = always from global memory.  Same results */
  int hp_sweep;       /* arithmetic of the FP64-data sweeps that use cached local inverses:
                         0 = automatic: float pairs in the FP64 phase of BGK_MIXED, FP64 otherwise;
                         1 = FP64; 2 = float pairs: the mass-weighted source, the inflow terms
                         and the product with the inverse (stored as float pairs) in
                         compensated FP32 arithmetic (error-free transformations), about
                         2^-44 relative per operation (FP64: 2^-53), eight orders below the
                         Picard tolerance, at a fraction of B300's FP64 instruction cost.
                         The data in memory stay FP64 */
  int refine;         /* BGK_MIXED: 0 = after the first FP64-phase sweep of a stage, every
                         further Picard iteration f <- f + d solves for the change d with an
                         FP32 sweep whose source is the change of nu M, whose wall data and
                         lagged inflow are those of the previous change and whose inflow data
                         are zero (exact in exact arithmetic: the iterate just swept satisfies
                         the sweep's equations, so the next sweep differs from it only through
                         these changes); with the projected Maxwellian the change of nu M
                         comes from the FP32 derivative of the projected factors at the
                         midpoint of the two iterates' primitive variables (about 1e-6 of the
                         change; a node whose variables changed by more than 1e-5 relative
                         takes the difference of both states' FP64 factors instead);
                         1 = every FP64-phase iteration a full sweep */
  int stage_predictor; /* multi-stage DIRK steps: 1 = each stage after the first starts its
                         Picard iteration from moments extrapolated across the stage
                         abscissae (U_k + dt sum_r A_sr G_r + dt A_ss G_{s-1}, G_r the moment
                         rate the earlier stages imply; the collision term conserves the
                         moments, so they move by transport only) instead of the previous
                         stage's moments; a node whose extrapolated density or temperature is
                         not positive keeps the previous stage's moments.  Changes where the
                         iteration starts, not its fixed point; 0 = off (the previous stage's
                         moments, as the paper's iteration) */
} bgk_config;

typedef struct {
  int n_stages;
  int iterations[3];  /* Picard iterations of each stage of the last step */
  double measure[3];  /* final convergence measure of each stage */
  int total_sweeps;   /* sweeps run since the handle was created */
  int status;
  int iterations_fp32[3];  /* BGK_MIXED: FP32-phase iterations of each stage (else 0) */
} bgk_stats;

typedef struct bgk_handle bgk_handle;

/* Build geometry, element tables, velocity grid and every ordinate's sweep graph
 * (generations by longest path, cycles broken by the DFS back-edge rule of Sec. 4.1)
 * on the current CUDA device, and allocate the state.  Errors: BGK_E_INVALID (bad
 * sizes, non-conforming or degenerate mesh), BGK_E_OOM, BGK_E_CUDA. */
int bgk_create(const bgk_mesh* mesh, const bgk_vgrid* vgrid, const bgk_physics* phys,
               const bgk_config* cfg, bgk_handle** out);
int bgk_destroy(bgk_handle* h);

/* Problem sizes: out[0]=n_ordinates, [1]=n_nodes, [2]=n_dof, [3]=n_cells, [4]=dim,
 * [5]=max generations over ordinates, [6]=lagged edges over all ordinates,
 * [7]=bytes of the local-inverse cache (0 if none), [8]=threads per sweep CTA,
 * [9]=sweep algorithm in use (1 TGS, 2 TS).  out holds 10 values. */
int bgk_sizes(const bgk_handle* h, int64_t* out);
/* Slots of the shared-memory front that the handle's generation sweeps use: its FP32
 * sweeps' (the FP32 shadow's with BGK_MIXED) or, for an FP64 handle, its float-pair sweeps'
 * (bgk_config.sweep_front, hp_sweep); 0 when they read every upwind trace from global
 * memory. */
int bgk_front_slots(const bgk_handle* h, int* slots);
/* Whether the mixed precision's FP64 phase uses the Picard refinement (bgk_config.refine):
 * *on = 1 when its iterations after the first of a stage are FP32 correction sweeps, else 0. */
int bgk_refine_active(const bgk_handle* h, int* on);
/* Time step actually used (after the CFL rule). */
int bgk_get_dt(const bgk_handle* h, double* dt);

/* Initial state f = nodal-in-x, projected-in-v Maxwellian (Sec. 3.3, App. B) of the
 * given nodal states (host [n_nodes][d+2]).  Resets the BDF2 history. */
int bgk_set_state_maxwellian(bgk_handle* h, const double* h_nut);
/* Inflow boundary data: projected Maxwellian of the nodal states (host [n_nodes][d+2]),
 * used at nodes of boundary faces with v.n < 0 (Eq. bgk-bc, inflow condition). */
int bgk_set_inflow_maxwellian(bgk_handle* h, const double* h_nut);
/* Inflow boundary data f^bc of Eq. bgk-bc given directly: host FP64 [n_ordinates][n_nodes]
 * (values at nodes not on a boundary face are ignored).  Copied; the caller keeps h_f.
 * BGK_E_INVALID on a null argument. */
int bgk_set_inflow(bgk_handle* h, const double* h_f);
/* Raw distribution in or out, host buffers [n_ordinates][n_nodes] of dtype. */
int bgk_set_f(bgk_handle* h, const void* h_f, int dtype);
int bgk_get_f(bgk_handle* h, void* h_f, int dtype);
/* Device-pointer variants (same layout), ordered on the handle's stream. */
int bgk_set_f_device(bgk_handle* h, const void* d_f, int dtype);
int bgk_get_f_device(bgk_handle* h, void* d_f, int dtype);
/* Overlapped input of the next state: bgk_upload_f_async starts copying host h_f ([n_ordinates]
 * [n_nodes] in the handle's storage type: BGK_DTYPE_F64 unless the precision is
 * BGK_FP32_SWEEP) into a staging buffer of the handle on a copy stream of its own and
 * returns at once; the copy may overlap the steps already queued.  h_f should be pinned
 * (page-locked) for the copy to run asynchronously and must stay valid and unchanged until
 * the next bgk_set_f_uploaded returns.  bgk_set_f_uploaded makes the state the staged one,
 * as bgk_set_f does, ordered after the copy on the handle's stream, without waiting on the
 * host.  A second upload before the staged state is taken waits (on the device) for that
 * hand-over.  BGK_E_INVALID: null arguments, the other dtype, or no upload pending;
 * BGK_E_OOM: no room for the staging buffer. */
int bgk_upload_f_async(bgk_handle* h, const void* h_f, int dtype);
int bgk_set_f_uploaded(bgk_handle* h);

/* Velocity moments of the current f, host [n_nodes][d+2] (Eq. moments). */
int bgk_get_moments(bgk_handle* h, double* h_U);
int bgk_get_moments_device(bgk_handle* h, double* d_U);
/* Ordinates and quadrature weights, host [n_ordinates][dim] and [n_ordinates]. */
int bgk_get_velocity(const bgk_handle* h, double* h_v, double* h_w);
/* Generation of every cell for ordinate j (host int32 [n_cells]); returns the count of
 * generations in *n_gen.  Bit-exact definition: longest path from a source (Sec. 4.1). */
int bgk_get_generations(bgk_handle* h, int j, int32_t* h_gen, int* n_gen);

/* Lagged edges of ordinate j's sweep graph (Sec. 4.1: the DFS back edges removed to break
 * cycles; their upwind values are taken from the previous Picard iterate).  Writes up to
 * `cap` pairs (upwind cell, downwind cell) to h_edges ([n][2], host) and their number to
 * *n_lagged (the total, also when it exceeds cap).  An inflow face is lagged exactly when
 * its upwind cell does not have a smaller generation. */
int bgk_get_lagged_edges(bgk_handle* h, int j, int32_t* h_edges, int cap, int* n_lagged);

/* Checkpoint / resume.  bgk_save writes the time-stepping state -- f^n, f^{n-1} when the
 * BDF2 history is present, the step count, and the learned guess's moment history when a
 * network is attached -- to the file `path` (raw little-endian binary behind a header that
 * records the problem's sizes, velocity grid, nu, dt, storage type and a hash of the mesh
 * geometry, the collision model and the wall kinds).  bgk_load reads such a file into a
 * handle created for the same problem (same mesh, grid, nu, dt, integrator, collision
 * model, walls and storage precision; else BGK_E_IO) and replaces its state: the next
 * bgk_step is bit-identical to the one the saving handle would take, given the same inflow
 * data (these are not in the file: set them on the loading handle).
 * Returns BGK_E_IO when the file cannot be written/read or does not match.  A file whose
 * header does not match leaves the handle's state as it was; a file that matches but ends
 * early (or fails to copy) leaves the handle without a state: bgk_step then returns
 * BGK_E_INVALID until the next bgk_set_* call or successful bgk_load. */
int bgk_save(bgk_handle* h, const char* path);
int bgk_load(bgk_handle* h, const char* path);
/* Steps taken since the state was last set or loaded (bgk_set_*, bgk_load restores the
 * saved count) and the corresponding time steps * dt. */
int bgk_get_time(const bgk_handle* h, int64_t* steps, double* t);

/* One transport sweep of the Picard iteration, Eq. (bgk-ss-picard): f <- solution with
 * the Maxwellian of the current moments, source q = q_scale * f_q and collision nu_s.
 * f_q is the handle's stage base state (the state at the last bgk_set_* call or step).
 * nu_s <= 0 / q_scale <= 0 select the first stage's values nu + 1/(dt A_11) and
 * 1/(dt A_11), for which the local-inverse cache (if any) was built.
 * For parity tests and sweep benchmarks; a step does not use this entry point. */
int bgk_sweep(bgk_handle* h, double nu_s, double q_scale);

/* Ordinate shards (Sec. 4: the sweeps of different ordinates are independent given the
 * Maxwellian of the current moments and the lagged values; the one coupling per Picard
 * iteration is the sum over ordinates in Eq. moments).  A sharded iteration over S parts of
 * the ordinates is: every part computes its partial moments, the parts' partial moments
 * are summed in a fixed order (an allreduce across devices), and every part sweeps its
 * ordinates with the summed moments.
 *   bgk_sweep_range: one sweep of the ordinates [j_begin, j_end) with the source built
 *     from the moments d_U (device, [node][d+2], the summed moments of the current
 *     iterate) and the handle's stage source, as bgk_sweep (nu_s, q_scale <= 0: the step's
 *     first-stage values).  Ordinates outside the range are not touched.  Returns
 *     BGK_E_NONPHYSICAL if d_U has n <= 0 or theta <= 0 somewhere, BGK_E_INVALID if the
 *     problem has bounce-back or reflecting walls (their mirror ordinates may lie in
 *     another part; the shards exchange no boundary data).
 *   bgk_moments_range_device: the partial moments of the current f over the ordinates
 *     [j_begin, j_end) into d_U (device, [node][d+2]); j_begin and j_end must be multiples
 *     of N^(d-1) (whole values of the outermost velocity index), else BGK_E_INVALID.
 *     The parts' partial moments add up to bgk_get_moments_device. */
int bgk_sweep_range(bgk_handle* h, int j_begin, int j_end, const double* d_U, double nu_s, double q_scale);
int bgk_moments_range_device(bgk_handle* h, int j_begin, int j_end, double* d_U);

/* The rest of a sharded step, so that the caller only orders calls and moves partial
 * moments between devices (Sec. 3.5 stages, Sec. 4 Picard loop):
 *   bgk_shard_step_begin(h, &S, &tol): f^k <- f (BDF2 after its start-up step: the stage
 *     source (4 f^n - f^{n-1}) / (2 dt) and the history); S = stages of this step, tol =
 *     tau / max(1, nu dt), the Picard tolerance of Eq. (convergence-criteria).
 *   for s < S: bgk_shard_stage_begin(h, s) -- stage s's source q^(s) (Eq. q-stages) and
 *     coefficient nu + 1/(dt A_ss); until the measure is below tol: partial moments
 *     (bgk_moments_range_device) summed over all parts in a fixed order
 *     (bgk_sum_partials_device after gathering), bgk_sweep_range with nu_s = q_scale = 0
 *     (the open stage's values), the new summed moments, bgk_conv_measure_device; then
 *     bgk_shard_stage_end(h, s) -- the stage derivative F_s (Eq. dirk-recursive-def).
 *   bgk_shard_step_end(h): f^{k+1} = f^k + dt sum_s b_s F_s (Eq. dirk-n) unless the method
 *     is stiffly accurate; the BDF2 history after the start-up step; the step count.
 * Every part holds the whole problem on its device and only its ordinates' values are
 * meaningful; given the same summed moments every part computes the same measure, so all
 * stop at the same iteration.  FP64 or FP32 handles without walls (BGK_MIXED and wall
 * coupling are not sharded): BGK_E_INVALID otherwise, or when called out of order.
 *   bgk_sum_partials_device: d_U = sum of n_parts arrays [node][d+2] stored one after
 *     another at d_parts, added in part order 0, 1, ... (the same bits on every device).
 *   bgk_conv_measure_device: *measure (host) = max(|dU_0|/|U_0|, |dU_1..d|/max(|U_1..d|,
 *     |U_0|), |dU_d+1|/|U_d+1|) of device moments d_U_new against d_U_old, l2 over nodes,
 *     summed in a fixed order (Eq. convergence-criteria with the design's reading for a
 *     zero momentum).  Allocates a small scratch; synchronizes the handle's stream. */
int bgk_shard_step_begin(bgk_handle* h, int* n_stages, double* tol);
int bgk_shard_stage_begin(bgk_handle* h, int stage);
int bgk_shard_stage_end(bgk_handle* h, int stage);
int bgk_shard_step_end(bgk_handle* h);
int bgk_sum_partials_device(const bgk_handle* h, const double* d_parts, int n_parts, double* d_U);
int bgk_conv_measure_device(bgk_handle* h, const double* d_U_new, const double* d_U_old, double* measure);

/* Advance nsteps implicit steps (Sec. 3.5 stages, Sec. 4 Picard loop to tolerance).
 * Each step runs as one CUDA graph with one conditional while-loop per stage.  st may
 * be NULL.  Errors: BGK_E_INVALID (no state set), BGK_E_NOCONV, BGK_E_NONPHYSICAL,
 * BGK_E_CUDA. */
int bgk_step(bgk_handle* h, int nsteps, bgk_stats* st);
/* Same, host-synchronous only at the end; returns immediately after enqueueing when
 * async != 0 (stats then come from bgk_last_stats after a stream sync). */
int bgk_step_async(bgk_handle* h, int nsteps);
int bgk_last_stats(bgk_handle* h, bgk_stats* st);
/* Make the handle's stream wait for completion. */
int bgk_synchronize(bgk_handle* h);

/* Instrumentation: the sweep kernel's event-timed average duration (ms) and launch
 * count since the last reset, recorded on the handle's stream. */
int bgk_timing(bgk_handle* h, int reset, double* sweep_ms_total, int64_t* sweep_launches);

/* Measured FMA rate of the current device in TFLOP/s (2 flops per fused multiply-add),
 * dtype BGK_DTYPE_F64 or BGK_DTYPE_F32: the best of three event-timed launches of
 * independent FMA chains on every SM (after one warm-up launch), on a stream of its own.
 * It is the denominator of the arithmetic roofline of the FP64 sweeps, whose local solves
 * are bound by the FP64 pipe (no FP64 tensor path is used).  Allocates and frees a few KB
 * of device memory.  Errors: BGK_E_INVALID, BGK_E_OOM, BGK_E_CUDA. */
int bgk_probe_fma_tflops(int dtype, double* tflops);

/* Choose the sweep algorithm by measurement (Sec. 4.1: TS wins when generations are narrow
 * and the ordinates many, TGS otherwise): times `reps` sweeps of each on the current state
 * (which must have been set; it is restored) with the first stage's coefficients, keeps
 * the faster and captures the step graphs again.  With BGK_MIXED the FP32 shadow chooses
 * for itself the same way.  ms (may be NULL) receives 4 values: TGS and TS time per sweep
 * of the main problem, then of the FP32 shadow (0 without one).  BGK_E_INVALID if no state
 * was set or reps <= 0. */
int bgk_autotune_sweep(bgk_handle* h, int reps, double* ms);

/* ---- Batched instances ---------------------------------------------------------------
 * Many independent problems (own mesh, velocity grid, nu, dt; backward Euler) advanced
 * together.  Per Picard iteration the sweeps of all instances run as one persistent
 * kernel over (instance, ordinate-block) units; each instance's Picard loop ends on its
 * own criterion (Eq. convergence-criteria) and finished instances skip their work; one
 * CUDA graph (a conditional while-node) covers a whole step.  Results of each instance
 * are identical to a single-instance run of the same configuration.  Arrays meshes,
 * vgrids, phys have n entries; cfg applies to all (its stream is shared).  Errors as
 * bgk_create; BGK_E_INVALID if an integrator is not BGK_BE. */
typedef struct bgk_batch bgk_batch;
int bgk_batch_create(int n, const bgk_mesh* meshes, const bgk_vgrid* vgrids, const bgk_physics* phys,
                     const bgk_config* cfg, bgk_batch** out);
int bgk_batch_destroy(bgk_batch* b);
/* The handle of instance i (owned by the batch; use it for bgk_set_*, bgk_get_*). */
int bgk_batch_instance(bgk_batch* b, int i, bgk_handle** h);
/* Autotuner: for each instance class (element type, ordinates, log2 cells) time the
 * batched sweep with 1, 2 and 4 ordinates per CTA (128, 64, 32 threads per ordinate)
 * over reps launches and keep the fastest (cached per class for the process); f is
 * restored afterwards.  h_block (optional, n entries) receives the choice. */
int bgk_batch_autotune(bgk_batch* b, int reps, int32_t* h_block);
/* nsteps steps of every instance; h_iters / h_status (optional, n entries) receive the
 * Picard iterations (FP32 + FP64 phases) and status of each instance's last step.
 * With cfg.precision = BGK_MIXED every step runs a batched FP32 phase over all
 * instances, then the batched FP64 phase.  Returns the first error. */
int bgk_batch_step(bgk_batch* b, int nsteps, int32_t* h_iters, int32_t* h_status);
/* One batched sweep of all instances (Maxwellian of the current moments, q = f^k/dt),
 * event-timed; bgk_batch_timing returns the accumulated time and launch count. */
int bgk_batch_sweep(bgk_batch* b);
int bgk_batch_timing(bgk_batch* b, int reset, double* sweep_ms_total, int64_t* sweep_launches);
/* out[0] = instances, [1] = total DOF (sum of n_ordinates * n_nodes), [2] = sweep units,
 * [3] = CTAs of the persistent sweep. */
int bgk_batch_info(const bgk_batch* b, int64_t* out);

/* ---- Learned initial guess (an addition beside the paper's method) ------------------
 * A multilayer perceptron F -> H -> H -> H -> O (tanh on the hidden layers, inputs and
 * outputs normalised column-wise) predicts, for every spatial node, the change of
 * q = (log n, u, log theta) over a stage from features of the stage-start moments, as a
 * correction to repeating the previous stage's change (the last feature block).  With
 * a network attached (bgk_set_guess), each stage's iterate 0 takes the predicted moments
 * (nodes with a non-physical prediction keep their own); the Picard loop of Sec. 4 then
 * runs to the usual criterion, so the converged state is the solver's, not the network's.
 * Parameters, host or device float arrays, flat in the order W0 [H][F], b0 [H], W1 [H][H],
 * b1, W2 [H][H], b2, W3 [O][H], b3 [O]; normalisation [mu_x (F), sd_x (F), mu_y (O),
 * sd_y (O)].  Training runs in FP32 on the current device's default stream; attached
 * networks run with BF16-stored weights and FP32 accumulation inside the step graph.
 * A network's scratch is shared: do not run two handles with the same network at once.
 * F, H, O <= 128.  Features per node (d = dimension, s = sqrt(theta)): q | s dt grad log n |
 * dt grad u | s dt grad log theta | log10(nu dt) | change of q over the previous stage. */
typedef struct bgk_mlp bgk_mlp;
int bgk_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, bgk_mlp** out);
int bgk_mlp_destroy(bgk_mlp* m);
int bgk_mlp_num_params(const bgk_mlp* m, int64_t* n);
int bgk_mlp_get_params(const bgk_mlp* m, float* h_params, float* h_norm);
int bgk_mlp_set_params(bgk_mlp* m, const float* h_params, const float* h_norm);
/* normalisation from data: column means and standard deviations of d_X [n][F], d_Y [n][O] */
int bgk_mlp_fit_norm(bgk_mlp* m, const float* d_X, const float* d_Y, int64_t n);
/* mean squared error on normalised outputs and its gradient (h_grad: host, optional) */
int bgk_mlp_loss_grad(bgk_mlp* m, const float* d_X, const float* d_Y, int64_t n, double* loss, float* h_grad);
/* one Adam step (beta 0.9, 0.999, eps 1e-8) on the batch; *loss is before the step */
int bgk_mlp_train_step(bgk_mlp* m, const float* d_X, const float* d_Y, int64_t n, float lr, double* loss);
/* de-normalised outputs d_Y [n][O]; bf16 != 0 uses BF16-stored weights */
int bgk_mlp_predict(bgk_mlp* m, const float* d_X, int64_t n, float* d_Y, int bf16);
/* feature and output counts of the handle's network: F = guess features, O = dim + 2 */
int bgk_guess_dims(const bgk_handle* h, int* n_features, int* n_outputs);
/* features of the current state into d_X [n_nodes][F] (device); records the history */
int bgk_guess_features(bgk_handle* h, float* d_X);
/* training targets: change of q from d_Ustart (device moments) to the current moments,
 * minus the previous change recorded in the stage-start features d_X */
int bgk_guess_targets(bgk_handle* h, const double* d_Ustart, const float* d_X, float* d_Y);
/* attach (or with NULL detach) a network; its current parameters are copied to BF16 */
int bgk_set_guess(bgk_handle* h, bgk_mlp* m);

/* Attach (NULL detaches) one guess network to every instance of a batch; the guesses run
 * one instance after another inside the batch's step graph. */
int bgk_batch_set_guess(bgk_batch* b, bgk_mlp* m);

/* Moments and convergence measure with no device allocation.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc, such as
 * programs that have given all device memory to their own pool allocator up front,
 * or programs that must never synchronize the device (cudaMalloc/cudaFree may).
 *
 * Computes, from d_f ([n_ordinates][n_nodes] of dtype on the current device), the
 * moments d_U_new ([n_nodes][dim+2], FP64) and writes to d_measure (one device double)
 * max(|dU_0|/|U_0|, |dU_1|/max(|U_1|, |U_0|), |dU_2|/|U_2|) against d_U_old -- the same
 * reduction and measure as the handle's Picard loop (FP32 data are summed in FP64 here and
 * as compensated float pairs by the handle: the two agree to 1e-12 relative, like FP64
 * data).  Work is enqueued on `stream`
 * (a cudaStream_t; NULL = the legacy default stream); results are ready when the
 * stream reaches that point.  Scratch lives in one file-scope device array of
 * 16384 x 6 doubles (768 KiB) that every GPU loading the library holds until exit:
 * n_nodes above 2,097,152 is rejected with BGK_E_INVALID.  Every call shares that
 * array and each call overwrites the rows it reads, so nothing has to start at zero;
 * calls that overlap on the GPU (two streams, or two host threads) race on it.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and should come before any stream capture.  Errors: BGK_E_INVALID, BGK_E_CUDA. */
int bgk_moments_measure_noalloc(const bgk_vgrid* vgrid, int dim, int64_t n_nodes, const void* d_f, int dtype,
                                const double* d_U_old, double* d_U_new, double* d_measure, void* stream);

const char* bgk_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* BGK_B300_H */
