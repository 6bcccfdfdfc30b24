/*
 * ap.h -- C ABI of the GB300 analytic-pulse gather + relativistic Boris push.
 *
 * Method: Weichman et al., "Analytic pulse technique for computational
 * electromagnetics" (arXiv:2307.04843).  The fields are split into an
 * analytic vacuum part E1/B1 and a grid part E2/B2 (Sec. 2, Eqs. E_1, E_2);
 * here each macroparticle evaluates E1/B1 in closed form at its own position
 * and time, adds the trilinearly gathered grid field (Sec. 2.1, Fig. 1: the
 * particle is pushed with the sum of the analytic and grid fields at its
 * position), and takes a relativistic Boris step.
 *
 * Units are normalised: c = omega0 = k0 = 1 (lambda = 2 pi), fields in
 * m c omega0 / e so that the field amplitude is a0 (Sec. 2.2, definition of
 * a0 under Fig. 3).  The particles are electrons, charge -1 and mass 1:
 *     du/dt = -(E + u x B / gamma),  dx/dt = u / gamma,  u = gamma beta.
 * The laser propagates along +z (the paper uses x):
 *     E_perp = Re[ Gamma(eta) u(x,y,z) p e^{i psi} ],
 *     psi    = omega (t - t_focus) - k (z - z_focus) + phase0,  k = omega / v_phi,
 *     eta    = (t - t_focus) - (z - z_focus) / v_g,
 *     B_perp = (B0/E0) z_hat x E_perp                      (Eqs. plane_func, plane_b).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: AP_OK (0) or a negative AP_ERR_*.
 *     The library never aborts, never prints and never traps the GPU.
 *   - All device memory passed in is owned and allocated by the caller; the
 *     library allocates only its handle and the handle's small parameter
 *     buffers (in ap_init_pulse), never on the push path.
 *   - Calls that take a stream are asynchronous and stream-ordered.  Errors
 *     found on the device (a non-finite particle state) are recorded in the
 *     handle's device status word and reported by ap_sync_status.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Particle state semantics (leapfrog): on entry x is at t0 and u at
 *     t0 - dt/2; after n_steps steps x is at t0 + n_steps dt and u at
 *     t0 + (n_steps - 1/2) dt.  The given u is taken as u^{-1/2} (no
 *     half-step back push).  Fields are sampled at t_n = t0 + n dt (computed,
 *     not accumulated) at the integer-step position x^n.
 */
#ifndef AP_H
#define AP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AP_ABI_VERSION 3

/* ------------------------------------------------------------ status codes */
#define AP_OK 0
#define AP_ERR_ARG -1        /* invalid argument (NULL pointer, bad size, bad enum) */
#define AP_ERR_ALIGN -2      /* a device pointer is not 16-byte aligned */
#define AP_ERR_CUDA -3       /* a CUDA runtime call failed */
#define AP_ERR_NONFINITE -4  /* a particle state or field became NaN/Inf */
#define AP_ERR_TIMEOUT -5    /* reserved: no entry point returns it.  No kernel of this library
                                waits on a flag, on another block or on another rank (every
                                loop is bounded by a count), so no device-side wait can expire */
#define AP_ERR_WORKSPACE -6  /* caller workspace too small */
#define AP_ERR_UNSUPPORTED -7 /* combination not built (e.g. Yee dispersion with a flying focus) */

/* ------------------------------------------------------------------ enums */
/* pulse kinds */
#define AP_PLANE 0        /* plane wave with envelope, Eqs. plane_func / plane_b (Sec. 2.1) */
#define AP_GAUSS 1        /* paraxial Gaussian beam, Eq. paraxial with D = 3 (Sec. 3.1) */
#define AP_LG 2           /* Laguerre-Gaussian LG_pl, named in Sec. 3.1 (textbook form) */
#define AP_FLYING_SUM 3   /* flying focus as a linear superposition of Gaussian spectral
                             components (Sec. 3.3) */
#define AP_FLYING_CF 4    /* closed-form Gaussian flying focus (Sec. 3.3, modified paraxial
                             limit): Eq. paraxial with x_f - x -> xi0 - xi, xi = z - v_f t,
                             x_R -> (1 - beta_f) x_R; focus at z_focus at t_focus, which is
                             also when the envelope peak is there; beta_f < 1 */
/* polarisation vector p */
#define AP_LIN_X 0        /* p = (1, 0) */
#define AP_LIN_Y 1        /* p = (0, 1) */
#define AP_CIRC_P 2       /* p = (1, -i): |E_perp| = a0 |u| Gamma, rotating */
#define AP_CIRC_M 3       /* p = (1, +i) */
/* temporal envelopes Gamma(eta) */
#define AP_ENV_SIN2 0     /* cos^2(pi eta / T) for |eta| <= T/2, T = 2 pi N / omega, N = env_len cycles */
#define AP_ENV_GAUSS 1    /* exp(-2 ln2 eta^2 / T^2), T = env_len = intensity FWHM */
#define AP_ENV_SGAUSS 2   /* exp(-(eta / tau)^(2 g)), tau = env_len, g = sg_order (Sec. 2.3) */
#define AP_ENV_CW 3       /* 1 */
/* flags */
#define AP_F_LONGITUDINAL 1u /* add E_z, B_z from div E = 0, div B = 0 (Sec. 3.1) */
#define AP_F_YEE_DISP 2u     /* second-order Yee v_phi, v_g, B0/E0 (Eqs. vphi, vg, e_amp) */
#define AP_F_1D3V 4u         /* reduced dimensionality (Sec. 3.2): the particles of this set
                                keep their transverse position (a 1-D line at that x, y in
                                the focusing pulse) while z and all three momentum
                                components advance (1D-3V) */
/* arithmetic of the push */
#define AP_FP64 0            /* everything in double; u arrays are double */
#define AP_FP32_PHASE64 1    /* fields and Boris in float; phase argument and position
                                accumulation in native double; u arrays are float */
#define AP_FP32_PHASEFF 2    /* as AP_FP32_PHASE64 but the phase argument and the position
                                are carried as float-float pairs (about 48-bit significand,
                                Dekker 1971 / Knuth TwoSum), so no FP64 instruction runs in
                                the step loop; u arrays are float, x arrays stay double */
/* adjoint objectives */
#define AP_OBJ_MEAN_GAMMA 0  /* J_s = (1/N_s) sum_{i in set s} gamma_i(T) */
/* differentiable parameters, in the order of dJ_dparams rows */
#define AP_NPARAM 4          /* d/d(a0, w0, z_focus, beta_f); beta_f is 0 except for flying focus */

/* -------------------------------------------------------------- structures */

/* Physical description of one pulse (one "pulse-parameter set").  The paper's
 * run-time parameters (Sec. 2.3: E0, omega, super-Gaussian order g, duration
 * tau, envelope delay, initial phase at a reference position) plus the beam
 * and flying-focus parameters of Secs. 3.1 and 3.3.  Host memory. */
typedef struct {
  int32_t kind;       /* AP_PLANE | AP_GAUSS | AP_LG | AP_FLYING_SUM */
  int32_t pol;        /* AP_LIN_X | AP_LIN_Y | AP_CIRC_P | AP_CIRC_M */
  int32_t env;        /* AP_ENV_*; ignored (CW) for AP_FLYING_SUM */
  int32_t sg_order;   /* super-Gaussian order g >= 1 */
  int32_t lg_p, lg_l; /* LG radial and azimuthal indices, 0 <= p <= 8, |l| <= 8 */
  int32_t n_comp;     /* flying focus: number of spectral components, 2..AP_MAX_COMP */
  uint32_t flags;     /* AP_F_* */
  double a0;          /* peak field amplitude: focal-plane peak of |u| for beams; for the
                         flying focus the peak on-axis envelope at mid-range (see kind) */
  double omega;       /* carrier frequency (1 = omega0) */
  double w0;          /* beam waist */
  double z_focus;     /* focal plane; flying focus: start z_a of the focal range */
  double t_focus;     /* time at which the envelope peak crosses z_focus; flying focus:
                         time t_a at which the focus is at z_a */
  double env_len;     /* see AP_ENV_* */
  double phase0;      /* carrier phase at (t_focus, z_focus) */
  double beta_f;      /* flying focus: focal velocity v_f / c (AP_FLYING_SUM: nonzero;
                         AP_FLYING_CF: below 1, may be negative) */
  double bw_frac;     /* flying focus: frequencies span omega (1 +- bw_frac) */
  double ff_length;   /* flying focus: length L of the focal range */
  double yee_dx, yee_dt; /* AP_F_YEE_DISP: cell size and time step of the Yee solver */
  double omega_p;     /* 0: vacuum.  > 0: plane wave in a linear cold plasma of plasma
                         frequency omega_p carrying the analytic current J1 (Sec. 4);
                         kind AP_PLANE only, envelope AP_ENV_GAUSS, AP_ENV_SGAUSS or
                         AP_ENV_CW.  k follows from omega^2 = omega_p^2 + c^2 k^2, or with
                         AP_F_YEE_DISP from the Yee relation with a leapfrog current
                         (Eq. dispersion_j, zeta = (omega dt/2)/sin(omega dt/2)) and
                         B0/E0 from Eq. e_amp_j; B carries the finite-duration terms of
                         Eq. b_corr_t and J1 those of Eq. j1 (Phi = 0).  AP_ERR_ARG if
                         omega is below the cut-off or the Yee relation has no real k. */
} ap_pulse_desc;

#define AP_MAX_COMP 128
#define AP_MAX_SETS 4096

/* Particle arrays (structure of arrays), device memory, caller-owned.
 * x, y, z: double in every precision.  ux, uy, uz: double for AP_FP64, float
 * otherwise.  Every pointer must be 16-byte aligned (AP_ERR_ALIGN otherwise).
 * The arrays are updated in place. */
typedef struct {
  double *x, *y, *z;
  void *ux, *uy, *uz;
  int64_t n;
  /* batched calls only: set s owns particles [set_offsets[s], set_offsets[s+1]);
   * device memory, n_sets + 1 non-decreasing entries, set_offsets[0] = 0,
   * set_offsets[n_sets] = n. */
  const int64_t *set_offsets;
  int32_t n_sets;
} ap_particles;

/* Static node-centred grid field E2/B2 (Eqs. E_2, Sec. 2.1), device memory,
 * caller-owned.  Six float arrays f[0..5] = Ex, Ey, Ez, Bx, By, Bz, each
 * [nz][ny][nx] with x fastest; nodes at lo + i (hi - lo)/(n - 1).  Positions
 * outside [lo, hi] are clamped to the box.  n >= 2 along every axis; the
 * f[] arrays need 4-byte alignment, `packed` 16-byte alignment.
 * `packed` (nullable) is a copy made by ap_grid_pack in the layout named by
 * `packed_layout`:
 *   AP_PACK_NODES: [nz][ny][nx][8] floats (Ex, Ey, Ez, Bx, By, Bz, 0, 0: one
 *     32-byte sector per node); a cell refetch touches 8 sectors instead of
 *     24; used by every precision, f[] may then be NULL;
 *   AP_PACK_CELLS: [nz-1][ny-1][nx-1][48] floats, per cell and component the
 *     trilinear coefficients (a0..a7) of
 *       F = a0 + a1 wx + a2 wy + a3 wz + a4 wx wy + a5 wy wz + a6 wx wz + a7 wx wy wz
 *     (w the position inside the cell, 0..1), each computed in double from
 *     the corners and rounded once: one contiguous 192-byte record per cell,
 *     the components interleaved in pairs (Ex, Ey), (Ez, Bx), (By, Bz):
 *     float 16 p + 2 k + h of a record is a_k of component 2 p + h.  The
 *     float pushes read it (7 FMA per component, two components per packed
 *     FMA), the FP64 push and the adjoint read f[], which must then be given. */
typedef struct {
  const float *f[6];
  int32_t nx, ny, nz;
  double lo[3], hi[3];
  const float *packed;
  int32_t packed_layout;
} ap_grid;

#define AP_PACK_NODES 0
#define AP_PACK_CELLS 1

/* Optional diagnostics, device memory, caller-owned; every pointer nullable.
 * Unless `accumulate` is nonzero the call zeroes the buffers it writes first. */
typedef struct {
  double *lightfront_max; /* [n_steps]: max over particles of |(gamma - u_z) - h0| after
                             each step, h0 = gamma - u_z on entry (plane-wave invariant) */
  uint32_t *gamma_hist;   /* [hist_bins]: final gamma, computed in double from the stored
                             u; bin = floor((gamma - lo) * (bins / (hi - lo))) clamped to
                             [0, bins - 1]; non-finite gamma not counted */
  int32_t hist_bins;
  double hist_lo, hist_hi;
  double *set_gamma_sum;  /* [n_sets] (batched) or [1]: sum of final gamma per set */
  int32_t accumulate;
} ap_diag;

/* Yee-staggered grid that receives the analytic fields on its nodes
 * (grid-node form of the technique: Sec. 2.1 and Fig. 1 set E1/B1 on the
 * grid every step and add them to the internally advanced E2/B2).  Node
 * (i, j, k) sits at lo + (i d[0], j d[1], k d[2]); inside the cell the
 * components sit at the Yee offsets (in cells)
 *   Ex (1/2,0,0)  Ey (0,1/2,0)  Ez (0,0,1/2)  Bx (0,1/2,1/2)  By (1/2,0,1/2)  Bz (1/2,1/2,0).
 * An unused axis has n = 1 and d = 0 (a 1-D grid along z holds Ex on the
 * whole nodes and By on the half nodes).  f[c]: device [nz][ny][nx], x
 * fastest, caller-owned, float (f64 = 0) or double (f64 != 0), aligned to
 * the element size; a NULL component is skipped. */
typedef struct {
  void *f[6];
  int32_t nx, ny, nz;
  int32_t f64;
  double lo[3], d[3];
} ap_yee_grid;

/* Independent 1-D vacuum Yee lines (the internal field update of Sec. 2.1
 * for a wave along z): E[l][k] = E_x at z_k, B[l][k] = B_y at z_{k+1/2},
 * both at whole time levels; device [n_lines][nz], caller-owned, double for
 * AP_FP64 and float for AP_FP32_PHASEFF. */
typedef struct {
  void *E, *B;
  int32_t nz, n_lines;
  double dz, dt;
} ap_yee1d;

#define AP_YEE1D_MAX_NODES 12288  /* nodes per line: the line stays on chip (registers) */

/* 1-D lines with a linear cold-plasma current (Sec. 4), device memory,
 * caller-owned, [n_lines][nz] each, double for AP_FP64 and float for
 * AP_FP32_PHASEFF, aligned to the element size:
 *   E[l][k] = E_x at z_k, B[l][k] = B_y at z_{k+1/2}, both at whole time
 *   levels; J[l][k] = J_x at z_k at half time levels (on entry t0 - dt/2);
 *   wp2 (nullable) = omega_p^2 at z_k, [n_lines][nz]; NULL: omega_p^2 of
 *   the field `omega_p` on every node.
 * J stands for 4 pi J / c in the field units: Ampere's law reads
 * dE/dt = curl B - J and the current obeys dJ/dt = omega_p^2 E.
 * z_k = z0 + k dz places the nodes for the analytic fields (ap_apt1d_run). */
typedef struct {
  void *E, *B, *J;
  const void *wp2;
  int32_t nz, n_lines;
  double dz, dt;
  double omega_p;
  double z0;
} ap_line1d;

#define AP_LINE1D_MAX_NODES_F32 12288 /* nodes per float line (the line sits in shared memory) */
#define AP_LINE1D_MAX_NODES_F64 6144  /* nodes per double line */
#define AP_APT1D_MAX_NODES_F32 8192   /* nodes per float line of ap_apt1d_run (it also keeps
                                         three per-node phase constants in shared memory) */

/* Launch shape, chosen by the autotuner (0 = library default). */
typedef struct {
  int32_t block;          /* threads per block, multiple of 32, <= 1024 */
  int32_t blocks_per_sm;  /* persistent kernels: resident blocks per SM */
  int32_t grid_cache;     /* float pushes with a AP_PACK_CELLS grid: where a thread keeps its
                             particles' current cells, 0 shared memory (12 slots each,
                             cp.async refetch), 1 registers (48 registers each, load refetch),
                             2 with two particles per thread: the first particle's cell in
                             registers and the second's in shared memory (one particle per
                             thread: as 1) */
  int32_t pairs;          /* AP_FP32_PHASEFF pushes without a grid or with a AP_PACK_CELLS
                             grid: 1 = each thread carries two particles, every FP32 operation
                             of the field, the Boris step and the position packed (f32x2) over
                             the pair; 0 = one particle per thread.  Results do not depend on
                             the launch shape within either setting. */
  int32_t tile;           /* batched launch: particles per tile, a multiple of the particles
                             a block carries (block x (1 + pairs)); 0 = one block's worth */
} ap_launch_cfg;

typedef struct ap_handle_s *ap_handle;
typedef struct ap_graph_s *ap_graph;

/* ------------------------------------------------------------- entry points */

/* ABI version (AP_ABI_VERSION). */
int ap_version(void);

/* Human-readable text of a status code; static storage, never NULL. */
const char *ap_status_string(int status);

/* Pulse setup (host, once; row a1 of the hot path).  Validates `descs`
 * (host array of n_sets descriptions, 1 <= n_sets <= AP_MAX_SETS) and derives
 * every constant in FP64: Rayleigh range k w0^2/2, LG normalisation, the
 * flying-focus component table, and optionally the Yee v_phi, v_g, B0/E0 of
 * Eqs. vphi, vg, e_amp.  Allocates the handle and a device copy of the
 * derived parameters on the current device.  *out receives the handle (NULL
 * on error).  Errors: AP_ERR_ARG (bad description), AP_ERR_UNSUPPORTED,
 * AP_ERR_CUDA. */
int ap_init_pulse(const ap_pulse_desc *descs, int32_t n_sets, ap_handle *out);

/* Releases the handle and its device buffers (synchronises the device). */
void ap_destroy(ap_handle h);

/* Bytes of the packed grid copy in layout g->packed_layout (AP_PACK_NODES:
 * 32 per node; AP_PACK_CELLS: 192 per cell), 0 for a bad grid or layout. */
size_t ap_grid_packed_bytes(const ap_grid *g);

/* Writes the packed copy of g->f[] in layout g->packed_layout into `packed`
 * (device, caller-owned, ap_grid_packed_bytes(g) bytes, 16-byte aligned) on
 * `stream`.  The interpolated field is that of Sec. 2.1's grid; only the
 * layout (and, for AP_PACK_CELLS, the rounding of the coefficient form)
 * differs.  Errors: AP_ERR_ARG, AP_ERR_ALIGN, AP_ERR_CUDA. */
int ap_grid_pack(const ap_grid *g, float *packed, void *stream);

/* Sets the launch shape used by later calls on this handle (NULL restores
 * the defaults).  Errors: AP_ERR_ARG for an invalid shape. */
int ap_set_launch(ap_handle h, const ap_launch_cfg *cfg);

/* Evaluates the analytic E1/B1 of set `set` at n points (test and
 * inspection hook; Eqs. plane_func, plane_b, paraxial and the divergence
 * conditions of Sec. 3.1).  xyzt: device double [4][n] (x, y, z, t rows).
 * EB_out: device double [6][n] (Ex, Ey, Ez, Bx, By, Bz rows).  precision:
 * AP_FP64 evaluates in double; AP_FP32_* in the float arithmetic of the push
 * with the given phase arithmetic.  Errors: AP_ERR_ARG, AP_ERR_CUDA. */
int ap_eval_fields(ap_handle h, int32_t set, const double *xyzt, int64_t n, double *EB_out,
                   int32_t precision, void *stream);

/* Gather + push (rows a2-a11): advances every particle n_steps steps under
 * the analytic field of set 0 plus the gathered grid field `g` (nullable),
 * all steps fused in one launch with the particle held in registers.
 * p: see ap_particles (set_offsets ignored).  diag: nullable.
 * Errors: AP_ERR_ARG, AP_ERR_ALIGN, AP_ERR_CUDA (launch). */
int ap_gather_push(ap_handle h, const ap_particles *p, const ap_grid *g, double t0, double dt,
                   int64_t n_steps, int32_t precision, const ap_diag *diag, void *stream);

/* Scratch needed by ap_gather_push_batched (bytes; the tile-queue counter). */
size_t ap_batch_workspace_bytes(ap_handle h);

/* Batched persistent gather + push (row a12): set s of the handle drives
 * particles [set_offsets[s], set_offsets[s+1]).  One persistent launch of
 * (SM count x blocks_per_sm) blocks pops fixed-size particle tiles from a
 * global atomic counter kept in `workspace` (device, >= ap_batch_workspace_bytes,
 * 16-byte aligned, zeroed by the call on `stream`); the loop is bounded by the
 * tile count, no block waits on another.  p->n_sets must equal the handle's
 * set count.  diag->set_gamma_sum receives per-set sums of final gamma.
 * Calls sharing one workspace must not overlap on the GPU.
 * Errors: AP_ERR_ARG, AP_ERR_ALIGN, AP_ERR_WORKSPACE, AP_ERR_CUDA. */
int ap_gather_push_batched(ap_handle h, const ap_particles *p, const ap_grid *g, double t0,
                           double dt, int64_t n_steps, int32_t precision, const ap_diag *diag,
                           void *workspace, size_t ws_bytes, void *stream);

/* Size of the static scratch array used by ap_gather_push_batched_static. */
#define AP_STATIC_SCRATCH_BYTES 4096

/* Allocation-free variant of ap_gather_push_batched (the paper has no
 * counterpart: this is a library-interface convenience).  For callers that
 * cannot call cudaMalloc when they push -- for example a host application
 * whose own allocator has already reserved the GPU's memory, or a time loop
 * that must not risk a device synchronisation or an out-of-memory failure in
 * the middle of a step.  Instead of a caller workspace it uses a file-scope
 * static __device__ array of AP_STATIC_SCRATCH_BYTES bytes that every GPU
 * loading the library holds until the process exits; the caller still passes
 * the particle arrays, grid and diagnostics.  Arguments and results are those
 * of ap_gather_push_batched.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it with the identity of the device's
 *     CUDA context; a call in a new context of that device (after
 *     cudaDeviceReset, for instance) looks it up again.  Make the first call
 *     on a device, and the first after its context was re-created, before
 *     any stream capture.
 *   - Every call on a device shares the one array; the tile counter in it is
 *     zeroed by each call on `stream`, but calls that overlap on the GPU race
 *     on it and must be serialised by the caller.
 *   - Returns AP_ERR_WORKSPACE if the scratch the call needs
 *     (ap_batch_workspace_bytes) exceeds AP_STATIC_SCRATCH_BYTES; otherwise
 *     the errors of ap_gather_push_batched.  Calls no cudaMalloc or cudaFree. */
int ap_gather_push_batched_static(ap_handle h, const ap_particles *p, const ap_grid *g,
                                  double t0, double dt, int64_t n_steps, int32_t precision,
                                  const ap_diag *diag, void *stream);

/* Captures ap_gather_push_batched (its memsets and the persistent launch)
 * into a CUDA graph on `stream` (which must not be the legacy default
 * stream); every pointer is baked into the graph and must stay valid.
 * ap_graph_launch replays it on a stream.  Errors: as the batched call. */
int ap_batch_graph_create(ap_handle h, const ap_particles *p, const ap_grid *g, double t0,
                          double dt, int64_t n_steps, int32_t precision, const ap_diag *diag,
                          void *workspace, size_t ws_bytes, void *stream, ap_graph *out);
int ap_graph_launch(ap_graph gr, void *stream);
void ap_graph_destroy(ap_graph gr);

/* Workspace for ap_push_adjoint: one checkpoint of the state every
 * ckpt_every steps plus the tape of the recomputed segment, each for every
 * resident particle slot of the adjoint kernels (48 B per state, 768 slots
 * per SM), independent of n.  Returns 0 for invalid arguments. */
size_t ap_adjoint_workspace_bytes(ap_handle h, int64_t n, int64_t n_steps, int32_t ckpt_every);

/* Discrete adjoint of the gather + push (row a13): gradient of the per-set
 * objective J_s = (1/N_s) sum_i gamma_i(T) (AP_OBJ_MEAN_GAMMA) with respect to
 * the pulse parameters (a0, w0, z_focus, beta_f) of every set.  p0 holds the
 * initial state (unchanged by the call).  Runs the forward push storing
 * checkpoints every ckpt_every steps in `workspace`, then sweeps the segments
 * backwards, recomputing each from its checkpoint and back-propagating
 * through the Boris step and the analytic fields.  Per-set gradients are
 * reduced warp -> block -> FP64 atomics into dJ_dparams (device double
 * [n_sets][AP_NPARAM]) and J into J_out (device double [n_sets], nullable).
 * The call zeroes both.  The grid, if given, enters the forward trajectory
 * and the position adjoint.  precision: AP_FP32_PHASEFF or AP_FP64.  The
 * beta_f row is nonzero only for AP_FLYING_CF.
 * Errors: AP_ERR_ARG, AP_ERR_ALIGN, AP_ERR_WORKSPACE, AP_ERR_CUDA;
 * AP_ERR_UNSUPPORTED for AP_FLYING_SUM or another precision. */
int ap_push_adjoint(ap_handle h, const ap_particles *p0, const ap_grid *g, double t0, double dt,
                    int64_t n_steps, int32_t ckpt_every, int32_t objective, int32_t precision,
                    double *dJ_dparams, double *J_out, void *workspace, size_t ws_bytes,
                    void *stream);

/* Waits for `stream`, then returns and clears the handle's device status
 * word: AP_OK or AP_ERR_NONFINITE; AP_ERR_CUDA if the wait itself failed. */
int ap_sync_status(ap_handle h, void *stream);

/* Number of sets in the handle, or AP_ERR_ARG. */
int ap_num_sets(ap_handle h);

/* Analytic E1/B1 of set `set` at time t on the staggered nodes of `g`
 * (grid-node form, Sec. 2.1 and Fig. 1), each component at its own Yee
 * offset, E and B both at t (the scheme of Sec. 2.1 keeps B at whole steps).
 * accumulate = 0 stores E1/B1; nonzero adds them to what f[] holds (the
 * total field E1 + E2 that the push interpolates).  precision as for
 * ap_eval_fields; the result is rounded once to the array type.
 * Errors: AP_ERR_ARG (bad set, sizes < 1 or above 2^23 per axis or 10^12
 * nodes in all, negative or non-finite spacing), AP_ERR_ALIGN, AP_ERR_CUDA. */
int ap_eval_nodes(ap_handle h, int32_t set, const ap_yee_grid *g, double t, int32_t accumulate,
                  int32_t precision, void *stream);

/* Analytic current J1 of plane-wave set `set` (Sec. 4, Eq. j1 with Phi = 0;
 * zero for a vacuum pulse) at time t on the E nodes of `g`: f[0], f[1], f[2]
 * receive J_x, J_y, J_z at the Ex, Ey, Ez offsets (J stands for 4 pi J / c,
 * Ampere's law dE/dt = curl B - J); f[3..5] must be NULL.  The split form of
 * Sec. 4 takes J1 at the half steps, t = t_n + dt/2.  accumulate and
 * precision as for ap_eval_nodes.  Errors: those of ap_eval_nodes;
 * AP_ERR_ARG also for a set that is not a plane wave or a non-NULL f[3..5]. */
int ap_eval_current(ap_handle h, int32_t set, const ap_yee_grid *g, double t, int32_t accumulate,
                    int32_t precision, void *stream);

/* n_steps steps of the second-order Yee scheme in vacuum on every line of
 * `y`, in the three-substep form of Sec. 2.1 with r = dt/dz:
 *   B[k] -= (r/2)(E[k+1] - E[k])   k = 0 .. nz-2
 *   E[k] -= r (B[k] - B[k-1])      k = 1 .. nz-1
 *   B[k] -= (r/2)(E[k+1] - E[k])   k = 0 .. nz-2
 * E[0] and B[nz-1] are held fixed (the ends of the line).  Each product and
 * difference is rounded separately in the stated order (no fused
 * multiply-add).  All steps run in one launch, one block per line with the
 * line on chip: in registers, a few consecutive nodes per thread (double
 * lines longer than 6144 nodes: in shared memory).  precision: AP_FP64 (double arrays) or
 * AP_FP32_PHASEFF (float arrays).  Errors: AP_ERR_ARG (nz < 2 or above
 * AP_YEE1D_MAX_NODES, n_lines < 0, n_steps < 0), AP_ERR_ALIGN, AP_ERR_CUDA. */
int ap_yee1d_run(const ap_yee1d *y, int64_t n_steps, int32_t precision, void *stream);

/* n_steps steps of the Yee line with a linear cold-plasma current -- the
 * traditional simulation that Sec. 4 compares the analytic current with --
 * on every line of `y`, r = dt/dz, a_k = dt wp2[k]:
 *   B[k] -= (r/2)(E[k+1] - E[k])                 k = 0 .. nz-2
 *   J[k] += a_k E[k]                              k = 0 .. nz-1  (J^{n+1/2})
 *   E[k] = (E[k] - r (B[k] - B[k-1])) - dt J[k]   k = 1 .. nz-1
 *   B[k] -= (r/2)(E[k+1] - E[k])                 k = 0 .. nz-2
 * E[0] and B[nz-1] are held fixed.  Each product, sum and difference is
 * rounded separately in the stated order (no fused multiply-add); with
 * wp2 = 0 the result is that of ap_yee1d_run bit for bit.  All steps run in
 * one launch, one block per line with the line on chip: float lines of up
 * to 6144 nodes in registers (a few consecutive nodes per thread), longer
 * float lines and double lines in shared memory.
 * Errors: AP_ERR_ARG (nz < 2 or above AP_LINE1D_MAX_NODES_F32/_F64,
 * n_lines < 0, n_steps < 0, NULL arrays, non-finite or non-positive dz, dt,
 * negative or non-finite omega_p), AP_ERR_ALIGN, AP_ERR_CUDA. */
int ap_plasma1d_run(const ap_line1d *y, int64_t n_steps, int32_t precision, void *stream);

/* n_steps steps of the same lines in the split form of Sec. 4 (Eqs. E_1_j,
 * E_2_j): E, B hold the internally advanced E2, B2 and J the physical plasma
 * current, driven by the total field E1 + E2; the analytic E1 and current
 * J1 are those of pulse set `set` at (x, y) = (0, 0), z_k = z0 + k dz:
 *   B2[k] -= (r/2)(E2[k+1] - E2[k])
 *   J[k] += a_k (E1(z_k, t_n) + E2[k])
 *   E2[k] = (E2[k] - r (B2[k] - B2[k-1])) - dt (J[k] - J1(z_k, t_n + dt/2))
 *   B2[k] -= (r/2)(E2[k+1] - E2[k])
 * with t_n = t0 + n dt.  The total field is E1 + E2 (ap_eval_nodes on a
 * 1-D grid with the same nodes gives E1, B1).  E1 and J1 are evaluated in
 * every step in the kernel, in the precision's arithmetic (AP_FP32_PHASEFF:
 * float with the float-float carrier phase), so E2 only carries the part of
 * the field that the analytic pulse and current miss.  The pulse must be
 * linearly polarised along x (the line carries E_x, B_y).
 * Errors: those of ap_plasma1d_run; AP_ERR_ARG also for a bad set, a pulse
 * not polarised along x, and with AP_FP32_PHASEFF for 2 n_steps + 1 >= 2^24
 * or nz above AP_APT1D_MAX_NODES_F32. */
int ap_apt1d_run(ap_handle h, int32_t set, const ap_line1d *y, double t0, int64_t n_steps,
                 int32_t precision, void *stream);

#ifdef __cplusplus
}
#endif
#endif
