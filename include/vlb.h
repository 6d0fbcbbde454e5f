/*
 * vlb.h -- C ABI of libvlb, a GB300 (sm_103a) solver for the vielbein
 * finite-difference lattice Boltzmann method of Busuioc & Ambrus,
 * "Lattice Boltzmann models based on the vielbein formalism for the
 * simulation of flows in curvilinear geometries" (arXiv:1708.05944).
 *
 * The hot path is one TVD-RK3 stage (Sec. III.A, Eq. rk3) of the reduced
 * distributions f', f'' (Sec. IV.A, Eq. fred) over every (cell, momentum)
 * pair: chi-formulation WENO-5 advection (Secs. III.B-C, Eqs. chi_def,
 * flux_def, weno5_flux), the Hermite-projected momentum-derivative term
 * (Sec. IV.C, Eqs. df_K_H, dfp_K_H, df_K_hh, dfp_K_hh), BGK relaxation to the
 * truncated Hermite equilibrium (Sec. IV.D, Eqs. feq_red, eq_gak_H,
 * eq_gak_hh), the moment reduction (Eq. macro_red) and diffuse-reflection
 * walls whose density n_w balances the wall mass flux (Sec. III.E, Eq. nw).
 *
 * Conventions
 *  - m = k_B = 1.  Axis 0 of momentum space is the wall-normal one (p^R for
 *    circular Couette flow), axis 1 the tangential one (p^phi).
 *  - Populations are the weighted ones of Sec. IV.B,
 *    f_ij = w_i w_j f(p_i, p_j) / (omega(p_i) omega(p_j)), so moments are plain sums.
 *  - Distribution layout (host or device, as passed): contiguous
 *    [cell][field][i][j], field 0 = f', field 1 = f'', cell running over the
 *    instances of a context in order, i over nq0 axis-0 nodes, j over nq1
 *    axis-1 nodes; real type double (VLB_FP64) or float (VLB_FP32_BULK).
 *  - Every call returns a vlb_status; vlb_last_error() gives the message.
 *  - Calls run on the CUDA stream given at creation (a cudaStream_t passed as
 *    void*, NULL = legacy default stream).  Compute calls are asynchronous;
 *    read calls synchronise that stream.
 *  - The library owns the device memory it allocates and frees it in
 *    vlb_destroy.  Pointers passed in with on_device = 1 stay owned by the
 *    caller and are only read or written during the call.
 *  - Compute calls need a CUDA device; without one they return VLB_ERR_CUDA.
 *    Model and quadrature queries (vlb_parse_model, vlb_quadrature) run on
 *    the host only.
 */
#ifndef VLB_H
#define VLB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vlb_ctx vlb_ctx;

typedef enum {
  VLB_OK = 0,
  VLB_ERR_INVALID = -1,     /* argument out of range or malformed */
  VLB_ERR_UNSUPPORTED = -2, /* valid in the method but not built (e.g. > 32 nodes on an axis) */
  VLB_ERR_CUDA = -3,        /* CUDA runtime failure (message holds cudaGetErrorString) */
  VLB_ERR_NONFINITE = -4,   /* a moment or wall density came out NaN or Inf */
  VLB_ERR_TIMEOUT = -5,     /* a bounded device wait ran out; results of that call are invalid */
  VLB_ERR_STATE = -6        /* call not allowed in the context's current state */
} vlb_status;

typedef enum { VLB_FULL = 0, VLB_HALF = 1 } vlb_quad_kind;           /* H(N;Q) or HH(N;Q) */
typedef enum { VLB_FP64 = 0, VLB_FP32_BULK = 1 } vlb_precision;
typedef enum { VLB_BGK = 0, VLB_SHAKHOV = 1 } vlb_collision;
typedef enum { VLB_CHI = 0, VLB_FTILDE = 1, VLB_CARTESIAN = 2 } vlb_formulation;
typedef enum {
  VLB_TAU_KN_OVER_NT = 0, /* tau = Kn / (n T), Eq. (hydro_tau) and Eq. (canalie_tau) */
  VLB_TAU_AOKI = 1,       /* tau = sqrt(pi/8) Kn / n, Eq. (tau_aoki) */
  VLB_TAU_KN_OVER_N = 2   /* tau = Kn / n (Sec. VI.C and VI.G runs) */
} vlb_tau_mode;

/* Model HH(N;Q) x H(N;Q) of Eq. (model): per axis the quadrature kind, the
 * expansion order N of the equilibrium (0 <= N < Q, Eq. norder_limit) and
 * the order Q.  An axis has Q nodes (full range) or 2Q nodes (half range). */
typedef struct {
  int kind[2];
  int N[2];
  int Q[2];
} vlb_model;

/* Circular Couette grid (Sec. VI.A.1): n_cells cells between r_in < r_out,
 * equidistant when stretch_A == 0, else tanh-stretched per Eq. (eta_def) with
 * amplitude 0 < stretch_A < 1 and centre 0 <= stretch_delta <= 1.
 *
 * Slab: an instance may hold only the cells [cell_begin, cell_end) of that
 * grid (both 0: all n_cells cells; otherwise 0 <= cell_begin, cell_end <=
 * n_cells, at least 3 cells), with the geometry of the full grid.  An end of
 * the slab that is not r_in or r_out is a halo end: no wall there, its three
 * ghost cells are the neighbouring slab's cells, written with vlb_write_halo
 * before every stage (the WENO-5 stencils of Sec. III.C reach three cells
 * across an interface).  This is the domain decomposition of the radial
 * direction: each slab steps as the whole grid would, cell for cell. */
typedef struct {
  int n_cells;
  double r_in, r_out;
  double stretch_A, stretch_delta;
  int cell_begin, cell_end;
} vlb_couette_grid;

/* Gradually expanding channel grid (Sec. VII.A-B, H/2 = 1): n_lambda cells in
 * the wall-normal coordinate lambda in [0, 1], stretched as
 * lambda = tanh(eta) / stretch_A with eta equidistant (Eq. canalie_stretch),
 * times n_xi equidistant cells in xi in [xi_in, xi_out]; wall shape
 * phi(xi) of Eq. (canalie_phi) with parameter re_c. */
typedef struct {
  int n_lambda, n_xi;
  double xi_in, xi_out, re_c, stretch_A;
} vlb_channel_grid;

/* Wall of a Couette instance: tangential velocity u^phi (= Omega R) and temperature. */
typedef struct {
  double u_tangential;
  double T;
} vlb_wall;

/* Parse the paper's model notation, e.g. "HH(4;8)xH(4;20)" (Eq. model).
 * Returns VLB_ERR_INVALID for malformed strings or N >= Q. */
vlb_status vlb_parse_model(const char* text, vlb_model* out);

/* Nodes and weights of one axis (Sec. IV.B): full range -- roots of H_Q with
 * the Gauss weights of Eq. (w_H); half range -- the Q roots of h_Q followed by
 * their negatives, with the weights of Eq. (w_hh).  p and w are host arrays of
 * nq = Q or 2Q doubles, written in the node order used for populations. */
vlb_status vlb_quadrature(const vlb_model* model, int axis, double* p, double* w);

/* Nodes, weights and the force kernels of one axis as built by the library:
 * K[k*nq + k'] (Eqs. df_K_H / df_K_hh, d/dp f) and Kt[k*nq + k'] (Eqs.
 * dfp_K_H / dfp_K_hh, d/dp (p f)), nq*nq doubles each; any output may be
 * NULL.  Host only; lets callers check the library's tables. */
vlb_status vlb_axis_tables(const vlb_model* model, int axis, double* p, double* w, double* K, double* Kt);

/* Number of nodes of an axis (Q or 2Q); negative vlb_status on error. */
int vlb_axis_nodes(const vlb_model* model, int axis);

/* Create a context of n_inst independent circular Couette instances (chi
 * formulation, Sec. VI.A) sharing one model and precision.  grids, inner and
 * outer walls, kn and tau_mode are host arrays of n_inst entries.  Allocates
 * the distribution buffers (three RK3 copies) on the current device.  The
 * distribution starts as f_eq(n=1, u=0, T=1).  Errors: VLB_ERR_INVALID
 * (n_cells < 3, r_in >= r_out, kn <= 0, bad model),
 * VLB_ERR_UNSUPPORTED (more than 32 nodes on an axis), VLB_ERR_CUDA. */
vlb_status vlb_create_couette(const vlb_model* model, vlb_precision prec, int n_inst,
                              const vlb_couette_grid* grids, const vlb_wall* inner,
                              const vlb_wall* outer, const double* kn, const int* tau_mode,
                              void* cuda_stream, vlb_ctx** out);

/* Create a gradually expanding channel context (Sec. VII): the upper half of
 * the channel in the vielbein frame of Eq. (canalie_phat), Eq. (canalie_boltz)
 * in the chi form with the discrete connection coefficients of Sec. VII.A
 * and tau = Kn / (n T) (Eq. canalie_tau).  Boundaries: specular reflection at
 * lambda = 0, diffuse reflection at rest and temperature T0 at lambda = 1
 * with a zero-mass-flux density n_w per column (Eq. nw), and particle
 * reservoirs at both ends: populations entering the domain see
 * f_eq(n_in or n_out, (0, u^xi of the adjacent cell), T0), those leaving
 * see the adjacent cell (zeroth-order extrapolation); vlb_set_channel_flow_rate
 * replaces the reservoirs by the paper's flow-rate ends.  Cell (s, p) is cell
 * index p * n_lambda + s of the distribution layout.  Axis 0 must be half
 * range; the vielbein stage kernels exist for 16 x 12 and 8 x 4 nodes, other
 * velocity sets (up to 32 nodes per axis) run only the Cartesian-split
 * formulation (vlb_set_formulation; stepping before it is VLB_ERR_UNSUPPORTED);
 * n_lambda >= 3, n_xi >= 4 and a multiple of 4.  Starts at f_eq(1, 0, T0). */
vlb_status vlb_create_channel(const vlb_model* model, vlb_precision prec, const vlb_channel_grid* grid, double kn,
                              double n_in, double n_out, double T0, void* cuda_stream, vlb_ctx** out);

/* Launch shapes of a channel context's stage kernel, each CTA marching up
 * ts lambda rows of a strip of tp xi-columns with nt threads; returns their
 * number (0 for Couette contexts, negative on error).  Arrays may be NULL. */
int vlb_channel_variants(const vlb_ctx* ctx, int* ts, int* tp, int* nt, int max);

/* Force contraction of channel launch shape v: 1 on the tensor cores (single
 * precision, TF32 with hi/lo operand splits), 0 on the CUDA cores (packed
 * FP32x2, or FP64 in double precision); negative on error. */
int vlb_channel_variant_tensor_cores(const vlb_ctx* ctx, int v);

/* Total number of cells over all instances, nodes per cell (nq0 * nq1), and
 * the size in bytes of one distribution copy in the layout documented above. */
vlb_status vlb_sizes(const vlb_ctx* ctx, long long* total_cells, int* nvel, long long* f_bytes);

/* Overwrite the walls (host arrays of n_inst entries). */
vlb_status vlb_set_walls(vlb_ctx* ctx, const vlb_wall* inner, const vlb_wall* outer);

/* Set the Knudsen number and the relaxation-time convention of every instance
 * (Couette: tau = Kn/(n T), Aoki's sqrt(pi/8) Kn/n or Kn/n, vlb_tau_mode; the
 * paper uses the first for the Navier-Stokes comparisons, Sec. VI, and the
 * second for its Kn scans).  The channel relaxes with tau = Kn/(n T) (Sec. VII.C);
 * another mode there gives VLB_ERR_UNSUPPORTED.  Kn must be finite and > 0
 * (VLB_ERR_INVALID).  Takes effect from the next stage; synchronises the stream. */
vlb_status vlb_set_knudsen(vlb_ctx* ctx, double kn, int tau_mode);

/* Channel contexts only: densities of the inlet and outlet particle reservoirs
 * and their temperature T0, which is also the wall temperature.  The reservoirs
 * read the "pressure ratio" of the benchmark workload (see vlb_create_channel);
 * the paper's own flow-rate ends are vlb_set_channel_flow_rate.  Calling this
 * switches the ends (back) to reservoirs.  All three must be finite and > 0
 * (VLB_ERR_INVALID); a Couette context gives VLB_ERR_UNSUPPORTED.  Takes effect
 * from the next stage. */
vlb_status vlb_set_channel_reservoirs(vlb_ctx* ctx, double n_in, double n_out, double T0);

/* Collision term of every stage: VLB_BGK (Eq. BGK, the default) or VLB_SHAKHOV, the
 * extension the paper names in Sec. II.C: relaxation towards f_eq + (1 - Pr) G, G the
 * heat-flux part of Grad's 13-moment form for the cell's own heat flux q (both components;
 * p^z integrated out as in Sec. II; projected on the model basis axis by axis), so that q
 * relaxes at Pr / tau while n, u, T relax as with BGK; prandtl > 0 (2/3 for hard spheres).
 * Each stage then adds a second pass (moments of F_prev, then cc dt (1 - Pr) G / tau onto
 * the stage's output).  Needs expansion orders >= 3 on both axes (VLB_ERR_UNSUPPORTED);
 * Couette and channel contexts; not with vlb_step_static_scratch. */
vlb_status vlb_set_collision(vlb_ctx* ctx, int collision, double prandtl);

/* Formulation of the advection of a Couette context: VLB_CHI (the default; Eq.
 * boltz_couette_kom and its stretched form) or VLB_FTILDE, the conservative f~ formulation
 * the paper compares it with (Sec. VI.B, Eqs. boltz_couette_cons, boltz_couette_str_cons,
 * flux_cons_R, flux_cons_eta): F~ = sqrt(g) f is reconstructed by WENO-5 and differenced as
 * p (e_{s+1/2} F~_{s+1/2} - e_{s-1/2} F~_{s-1/2}) / d eta (e = 1, d eta = d R on the
 * equidistant grid), the walls act on F~ (Sec. III.E; n_w then carries sqrt(g)), and the
 * force term takes 1 / R at the cell centre.  It conserves sum d eta sqrt(g) sum f' exactly
 * but does not hold f = const at the walls (the paper's point).  The distribution stays f in
 * every call.  VLB_FTILDE runs on the fused stage kernel's f~ instance for velocity sets of
 * the fused path, with launch shapes 0 and 1 only (the first shape, plain and persistent;
 * switching selects one of them, vlb_set_variant refuses the others with VLB_ERR_INVALID and
 * vlb_autotune times those two), and on the multi-kernel stage for larger sets; not with
 * slabs or vlb_step_static_scratch.
 * Channel contexts: VLB_CHI (the vielbein stage of vlb_create_channel) or VLB_CARTESIAN, the
 * Cartesian-split channel the paper compares it with (Sec. VII.G, Eqs. canalie_coord_beq_cons,
 * canalie_coord_nw): the model's axes are read as the Cartesian momenta (p^x, p^y) (the
 * distribution and the moments of every call are then in that frame), there is no force
 * term, V^lambda = (p^x - lambda phi' p^y) / (1 + phi), V^xi = (1 + phi) p^y, the wall's
 * incoming half-plane V^lambda < 0 is taken per column, and the fluxes are of F itself (the
 * rest state is not an exact steady state of this scheme); reservoir ends only, no
 * post-processing (VLB_ERR_STATE).  Velocity sets with a vielbein kernel (16 x 12 and 8 x 4
 * nodes) run it on the same marching kernel and its launch shapes; others on a three-pass stage.  Errors: VLB_ERR_INVALID, VLB_ERR_UNSUPPORTED (f~ on a
 * channel, Cartesian on a Couette context), VLB_ERR_STATE. */
vlb_status vlb_set_formulation(vlb_ctx* ctx, int formulation);

/* Replace the channel's reservoirs by the paper's flow-rate ends (Sec. VII.C.1-2,
 * Eqs. canalie_inlet, canalie_outlet, canalie_inlet_s), half-channel particle flow
 * rate q0 >= 0 at both ends: per row s (lambda_s the row centre, H = 2) the
 * populations entering the domain see f_eq(n_s, (0, Q_s), T0) with
 * Q_s = 3 q0 (1 - lambda_s^2) / (H (1 + phi(xi_end))) and n_s fixed by the
 * particle flux through the end interface (entering part plus the leaving
 * populations of the adjacent cell) being (1 + phi) Q_s, i.e. Q_s in the
 * Cartesian frame; the leaving populations see the adjacent cell (zeroth
 * order).  T0 is the one of vlb_set_channel_reservoirs (default 1);
 * vlb_set_channel_reservoirs switches back.  Errors: VLB_ERR_INVALID (q0 < 0
 * or not finite), VLB_ERR_UNSUPPORTED (not a channel context). */
vlb_status vlb_set_channel_flow_rate(vlb_ctx* ctx, double q0);

/* Channel post-processing (Sec. VII.D-F) of the current state, in FP64 on the device:
 * ux, uy  -- the Cartesian velocity of Eq. (canalie_u) per cell (n_lambda n_xi, the
 *            cell order p * n_lambda + s of the distribution layout);
 * omega   -- the vorticity of Eq. (canalie_vorti) per cell, d/d xi by centred
 *            differences (second-order one-sided at the first and last column),
 *            d/d lambda by the paper's three-point formulas on the stretched rows;
 * psi     -- the stream function of Eq. (canalie_psi_sol) at the row interfaces,
 *            (n_lambda + 1) per column, index p * (n_lambda + 1) + s for
 *            lambda_{s}, zero on the centreline, x = lambda (1 + phi) spacing;
 * pw      -- the wall pressure per column: n T extrapolated linearly from the last
 *            two rows to the wall.
 * Host arrays; any may be NULL.  The normalised wall pressure of Eq.
 * (canalie_wall_pressure) is (pw - pw at the reference column) / (rho0 u0^2).
 * Errors: VLB_ERR_UNSUPPORTED (not a channel context), VLB_ERR_CUDA. */
vlb_status vlb_channel_postprocess(vlb_ctx* ctx, double* ux, double* uy, double* psi, double* omega, double* pw);

/* Set every cell of every instance to f_eq(n0, (u0, u1), T0) (Eq. feq_red). */
vlb_status vlb_init_equilibrium(vlb_ctx* ctx, double n0, double u0, double u1, double T0);

/* Copy a distribution in (vlb_set_f: becomes the current F_l) or out
 * (vlb_read_f: the most recently written one -- after vlb_stage(k) that
 * stage's output, after vlb_step the new F_l).  f has the documented layout
 * and the context's real type; on_device selects a device or host pointer.
 * The device buffers hold the deviation F - R from the rest state
 * R = f_eq(1, 0, 1) (populations w0_i w1_j): a kernel converts on the way in
 * and out, each element summed in double and rounded once.  A host copy is
 * staged in a distribution buffer that holds nothing live at the time. */
vlb_status vlb_set_f(vlb_ctx* ctx, const void* f, int on_device);
vlb_status vlb_read_f(vlb_ctx* ctx, void* f, int on_device);

/* One RK3 stage k in {1, 2, 3} (Eq. rk3) on the context buffers, with time
 * step dt (> 0: the same for all instances; 0: per-instance steps set by
 * vlb_set_dt).  Stage 1 reads F_l and writes F^(1); stage 2 reads F_l and
 * F^(1) and writes F^(2); stage 3 reads F_l and F^(2) and writes F_{l+1},
 * which then becomes the current distribution.  For parity tests. */
vlb_status vlb_stage(vlb_ctx* ctx, double dt, int k);

/* nsteps full TVD-RK3 steps (3 stages each), asynchronous on the stream. */
vlb_status vlb_step(vlb_ctx* ctx, double dt, long long nsteps);

/* nsteps full RK3 steps like vlb_step, but launched as a CUDA graph: three
 * steps (nine stage launches) are captured once per launch shape and
 * replayed nsteps / 3 times; the remaining steps are launched directly.
 * Results are identical to vlb_step.  The first call after a change of
 * launch shape captures (on the context stream, or on a private stream when
 * the context uses the legacy default stream), so make it before any
 * capture of your own. */
vlb_status vlb_step_graph(vlb_ctx* ctx, double dt, long long nsteps);

/* Run a Couette context towards its steady state: repeat (check_steps
 * graph-launched steps, then the L2 norms of Eq. msites_steady against the
 * previous check) until every instance has max(L2_u, L2_n, L2_T) < threshold
 * or max_steps steps were taken.  Reports the steps taken, each instance's
 * last residual and the step count at which it first fell below the
 * threshold (-1 if it never did); any output pointer may be NULL. */
vlb_status vlb_run_to_steady(vlb_ctx* ctx, double dt, long long check_steps, double threshold, long long max_steps,
                             long long* steps_taken, double* residual, long long* converged_step);

/* Per-instance time steps (host array of n_inst doubles > 0) used when dt = 0. */
vlb_status vlb_set_dt(vlb_ctx* ctx, const double* dt);

/* Macroscopic fields per cell (Eqs. macro_red): n, u^0, u^1, T, and optionally
 * T^{ab} (3 per cell: 00, 01, 11) and q^a (2 per cell), computed in FP64 from
 * the most recently written distribution (as for vlb_read_f).  Arrays hold total_cells (x3, x2) doubles; any
 * pointer may be NULL.  Synchronises the stream; VLB_ERR_NONFINITE if a
 * moment is NaN or Inf. */
vlb_status vlb_read_moments(vlb_ctx* ctx, double* n, double* u0, double* u1, double* T,
                            double* Tab, double* q, int on_device);

/* Wall densities n_w (Eq. nw) of the last stage: 2 per instance (inner, outer)
 * for Couette contexts (0 at a halo end of a slab), one per xi column for the
 * channel. */
vlb_status vlb_wall_density(vlb_ctx* ctx, double* nw);

/* Steady-state norms of Eq. (msites_steady) between the current moments and
 * those of the previous call (the first call only stores them and returns
 * zeros): per instance L2_u, L2_n, L2_T (host arrays of n_inst, NULL allowed). */
vlb_status vlb_residual(vlb_ctx* ctx, double* l2_u, double* l2_n, double* l2_T);

/* The squared norms of vlb_residual before the square root, per instance:
 * sum_s w_s (du_s / u_w)^2, sum_s w_s (n_s / n_prev,s - 1)^2 and the same for T,
 * over the instance's own cells.  Slabs of one grid add theirs (one
 * all-reduce of three numbers per instance) and take the square root.  Same
 * state rules as vlb_residual (the first call stores the moments). */
vlb_status vlb_residual_sums(vlb_ctx* ctx, double* s_u, double* s_n, double* s_T);

/* Slab halos (Couette contexts whose instances have halo ends, see
 * vlb_couette_grid).  A halo block is three cell rows in the library's
 * device form (the deviation from the rest state, fields interleaved per
 * velocity, rows padded): vlb_halo_bytes bytes, meaningful only to a context
 * of the same model and precision.
 *
 * vlb_read_edge copies the three cells at end `end` (0: the r_in side, cells
 * 0, 1, 2 of the instance; 1: the r_out side, its last three cells, in
 * increasing radius) of the distribution the next stage reads (the one
 * vlb_stage(ctx, dt, k) with k = the next stage number takes as F_prev) into
 * rows.  vlb_write_halo copies rows into the ghost cells of end `end` (0: the
 * three cells below the slab, in increasing radius; 1: the three above it).
 * Between the two, the caller moves the block to the neighbouring slab
 * (a device copy, or host or NCCL messages between processes).  A context
 * with a halo end steps with vlb_stage only: vlb_step, vlb_step_graph,
 * vlb_run_to_steady and vlb_step_static_scratch return VLB_ERR_STATE.
 * rows is host or device memory (on_device); the copy is complete when the
 * call returns.  Errors: VLB_ERR_INVALID (bad instance or end, null rows),
 * VLB_ERR_STATE (vlb_write_halo on an end that is a wall). */
long long vlb_halo_bytes(const vlb_ctx* ctx);
vlb_status vlb_read_edge(vlb_ctx* ctx, int inst, int end, void* rows, int on_device);
vlb_status vlb_write_halo(vlb_ctx* ctx, int inst, int end, const void* rows, int on_device);

/* Write / restore the distribution and step counter to / from a file
 * (little-endian; a header records model, precision and sizes, checked on load).
 * The file holds the device representation -- the deviation F - R from the
 * rest state in the context's real type -- so a run continued from it is
 * bitwise the run that wrote it. */
vlb_status vlb_save(vlb_ctx* ctx, const char* path);
vlb_status vlb_load(vlb_ctx* ctx, const char* path);

/* Launch shapes of the fused stage kernel available for this context: cells
 * per tile, threads per CTA and whether the launch is persistent (as many
 * CTAs as fit on the device, each walking the (instance, tile) list) or has
 * one CTA per tile; written to tc[], nt[], persistent[] (up to max entries,
 * NULL allowed).  Returns their number (negative vlb_status on error).  Every
 * shape computes the same stage; they differ in occupancy and load balance. */
int vlb_variants(const vlb_ctx* ctx, int* tc, int* nt, int* persistent, int max);

/* Select a launch shape by index (0 = default).  VLB_ERR_INVALID for an index out of range,
 * or above 1 while a Couette context runs the f~ formulation on the fused kernel. */
vlb_status vlb_set_variant(vlb_ctx* ctx, int variant);

/* Time every launch shape on this context's own workload (reps launches of
 * stage 1 each, with time step dt as in vlb_stage, CUDA events on the
 * context stream; stage 1 only writes scratch, so the distribution is
 * unchanged), keep the fastest and report its index and mean time per launch
 * (either pointer may be NULL). */
vlb_status vlb_autotune(vlb_ctx* ctx, double dt, int reps, int* chosen, double* best_ms);

/* nsteps (>= 1) TVD-RK3 steps of the instances of a circular Couette context
 * from the caller's device buffer f_in into the caller's device buffer f_out
 * (distinct, both in the documented layout and the context's real type; f_in
 * is only read), with a finite time step dt > 0 for every instance.  The paper
 * has no counterpart: this entry point is for callers that cannot allocate
 * device memory when they step (their memory belongs to another allocator or
 * to a full pool, or the step runs where cudaMalloc is not allowed).  It
 * allocates nothing: the two intermediate stage buffers F^(1), F^(2) live in
 * one static device array of 64 MiB compiled into the library (every GPU that
 * loads the library holds it until the process exits), so
 * 2 x total_cells x 2 x nvel x sizeof(real) must not exceed 64 MiB, else
 * VLB_ERR_UNSUPPORTED; nvel must be a multiple of 4, else VLB_ERR_UNSUPPORTED;
 * a channel context gets VLB_ERR_UNSUPPORTED and nothing is launched.  The
 * context's device must be the current device (else VLB_ERR_INVALID).  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), and a call whose dt differs from the context's
 * current time step copies the instance descriptors and synchronises the
 * stream (as vlb_set_dt does): make the first call, and any call that changes
 * dt, outside stream capture.  All calls share the array and it keeps the
 * last call's contents (nothing in it needs to start at zero): calls that
 * overlap on the GPU -- two streams, two contexts, or a context's own
 * vlb_step running concurrently -- race on it.  Asynchronous on the context
 * stream otherwise; it also updates the context's per-instance time step to
 * dt and its wall densities (vlb_wall_density). */
vlb_status vlb_step_static_scratch(vlb_ctx* ctx, const void* f_in, void* f_out, double dt, long long nsteps);

/* Measured double-precision FMA throughput of the current device in TFLOP/s
 * (2 flops per fma): the denominator of the roofline of the FP64 stage
 * kernels.  No counterpart in the paper.  Launches a timing kernel on the
 * default stream and allocates 8 bytes of device memory; about 0.1 s. */
vlb_status vlb_peak_fp64(double* tflops);

/* Number of kernels the last vlb_step / vlb_stage call launched. */
long long vlb_kernel_launches(const vlb_ctx* ctx);

/* Seed every cell of a context from macroscopic fields (host or device arrays
 * of total_cells doubles; q0 may be NULL, meaning zero).  The seed is Grad's
 * distribution with its heat-flux part only, the flux along axis 0,
 *   f = f_M(n, u, T) [1 + q0 xi_0 / (n T^2) (xi^2 / (5 T) - 1)],  xi = p - u,
 * reduced over p^z (Sec. II) and projected on the model's basis axis by axis
 * as the equilibrium of Sec. IV.D is; with q0 = 0 it is that truncated
 * equilibrium, f' = n g_0 g_1 and f'' = T f'.  When both expansion orders are
 * at least 3 the model moments of the seed return n, u, T and q0 exactly.
 * Host arrays are checked (finite, n > 0, T > 0; VLB_ERR_INVALID otherwise);
 * device arrays are used as given.  Synchronises the stream. */
vlb_status vlb_init_from_moments(vlb_ctx* ctx, const double* n, const double* u0, const double* u1, const double* T,
                                 const double* q0, int on_device);

/* ---- Learned warm start (no counterpart in the paper) -------------------
 * A 1D spectral neural operator over the normalised radius s in (0, 1) on
 * grid_points uniform points, mapping (Kn, inner wall speed, R_out/R_in) to
 * n, u^phi, T, q^R at every point.
 * Features per point: [(log10 Kn + 1)/2, (u_w - 0.255)/0.245, (R_out/R_in - 2.75)/1.25, 2s - 1].
 * Lift to `width` channels, then `layers` layers of h <- act(S(h) + h W + b)
 * (GELU, none on the last layer).  S is a truncated real DFT over `modes`
 * modes, a general real (2 width x 2 width) map per mode on its (Re, Im)
 * channel pair, and the inverse truncated DFT.  Projection: GELU(h P1 + c1) P2 + c2.
 * Parameters form one FP32 vector, ordered:
 *   W_in (4 x width), b_in (width),
 *   per layer: S (modes x 2width x 2width), W (width x width), b (width),
 *   P1 (width x hidden), c1 (hidden), P2 (hidden x 4), c2 (4);
 * matrices are [in][out], row-major.
 * GEMMs are BF16 tensor-core MMAs with FP32 accumulation.  Master weights
 * and the Adam state are FP32.  Outputs and targets are in physical units,
 * normalised inside by vlb_no_set_target_scaling.  cond arrays hold B rows
 * of (Kn, u_w, R_out/R_in); outputs and targets hold B x grid_points x 4
 * values.  The operator is resolution invariant: parameters trained at one
 * grid_points serve any other with 2 modes <= grid_points. */
typedef struct vlb_no vlb_no;
vlb_status vlb_no_create(int grid_points, int width, int modes, int layers, int hidden, void* cuda_stream,
                         vlb_no** out);
long long vlb_no_num_params(const vlb_no* no);
vlb_status vlb_no_set_params(vlb_no* no, const float* theta);  /* host array; resets the Adam state */
vlb_status vlb_no_get_params(vlb_no* no, float* theta);
vlb_status vlb_no_set_target_scaling(vlb_no* no, const double* mean4, const double* std4);
vlb_status vlb_no_predict(vlb_no* no, const double* cond, int B, double* out);
/* Mean squared error of the normalised outputs and its gradient (either output may be NULL). */
vlb_status vlb_no_loss_and_grad(vlb_no* no, const double* cond, const double* targets, int B, double* loss,
                                float* grad);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the batch; reports the loss before the step. */
vlb_status vlb_no_train_step(vlb_no* no, const double* cond, const double* targets, int B, double lr, double* loss);
const char* vlb_no_last_error(const vlb_no* no);
void vlb_no_destroy(vlb_no* no);

const char* vlb_last_error(const vlb_ctx* ctx);
void vlb_destroy(vlb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* VLB_H */
