/*
 * oracle.h -- plain, slow FP64 CPU oracle for the analytic-pulse field
 * evaluation + relativistic Boris push (Weichman et al., "Analytic pulse
 * technique for computational electromagnetics", arXiv:2307.04843).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code.  Only the tests, the package's smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no header, helper,
 * table or constant generator with the CUDA path: every derived constant
 * (Rayleigh range, Laguerre-Gaussian normalisation, flying-focus component
 * table, numerical-dispersion factors) is recomputed here from the physical
 * pulse description.
 *
 * Conventions (normalised units, c = omega0 = k0 = 1, lambda = 2 pi; fields in
 * m c omega0 / e so that the field amplitude is a0, Sec. 3.1 below Fig. 3):
 *   - propagation along +z (the paper propagates along x, Sec. 2.1);
 *   - E_perp = Re[ Gamma(eta) u(x,y,z) p e^{i psi} ],
 *     psi = omega (t - t_f) - k (z - z_f) + phase0  (Eq. plane_func),
 *     eta = (t - t_f) - (z - z_f) / v_g            (envelope argument);
 *   - B_perp = (B0/E0) z_hat x E_perp              (Eq. plane_b);
 *   - electron: q = -1, m = 1, du/dt = -(E + u x B / gamma), dx/dt = u/gamma;
 *   - plasma (Sec. 4): Ampere's law dE/dt = curl B - J, the usual sign.  Eq.
 *     E_1_j prints a plus sign, but with the current of Eq. j1 only the minus
 *     sign gives the dispersion relation Eq. dispersion_j (omega^2 = omega_p^2
 *     + c^2 k^2 in the continuum), so the plus is read as a misprint.
 *
 * Formulas are written in the textbook (w, R, atan Gouy) form with explicit
 * Laguerre sums; the longitudinal components come from 4th-order central
 * finite differences of the complex transverse profile (Sec. 3.1, the
 * divergence conditions below Eq. paraxial).
 *
 * Parity pins: none of the functions here is unpinned; the pinning tests are
 * tests/test_oracle_*.py.
 */
#ifndef APT_ORACLE_H
#define APT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* pulse kinds */
#define OR_PLANE 0   /* plane wave with envelope, Eq. plane_func / plane_b */
#define OR_GAUSS 1   /* paraxial Gaussian (LG_00), Eq. paraxial, D = 3 */
#define OR_LG 2      /* Laguerre-Gaussian LG_pl (named in Sec. 3.1, textbook form) */
#define OR_FLYING 3  /* flying focus as a sum of Gaussian spectral components (Sec. 3.3) */
#define OR_FLYING_CF 4 /* closed-form Gaussian flying focus (Sec. 3.3, modified paraxial limit) */

/* polarisations: p = (1,0), (0,1), (1,-i), (1,+i) */
#define OR_LIN_X 0
#define OR_LIN_Y 1
#define OR_CIRC_P 2
#define OR_CIRC_M 3

/* temporal envelopes Gamma(eta) */
#define OR_ENV_SIN2 0    /* cos^2(pi eta / T), |eta| <= T/2, T = 2 pi N / omega */
#define OR_ENV_GAUSS 1   /* exp(-2 ln2 eta^2 / T^2), T = intensity FWHM */
#define OR_ENV_SGAUSS 2  /* exp(-(eta/tau)^(2g)), Sec. 2.3 run-time parameters */
#define OR_ENV_CW 3      /* 1 */

#define OR_MAX_COMP 256

typedef struct {
  int kind, pol, env, sg_order;
  int lg_p, lg_l;
  int n_comp;        /* flying focus: number of spectral components */
  int longitudinal;  /* nonzero: add E_z, B_z from the divergence conditions */
  int yee;           /* nonzero: second-order Yee v_phi, v_g, B0/E0 (Eqs. vphi, vg, e_amp) */
  int one_d;         /* nonzero: 1D-3V push (Sec. 3.2), transverse position held fixed */
  double a0, omega, w0;
  double z_focus, t_focus;  /* focus position; time at which the envelope peak is there.
                               flying focus: start z_a of the focal range and its time t_a */
  double env_len;           /* SIN2: cycles N; GAUSS: intensity FWHM; SGAUSS: tau */
  double phase0;
  double beta_f;            /* flying focus: focal velocity v_f / c (closed form: < 1) */
  double bw_frac;           /* flying focus: half-width of the frequency spread / omega */
  double ff_length;         /* flying focus: length L of the focal range */
  double yee_dx, yee_dt;    /* cell size and time step entering Eqs. vphi, vg, e_amp */
  double omega_p;           /* nonzero: plane wave in a linear cold plasma of plasma frequency
                               omega_p, with the analytic current J1 of Sec. 4 (kind OR_PLANE,
                               Gaussian, super-Gaussian or CW envelope) */
} or_pulse;

typedef struct {
  or_pulse p;
  double k, vphi, vg, bratio;  /* wavenumber, phase/group velocity, B0/E0 */
  double zR;                   /* Rayleigh range k w0^2 / 2 */
  double amp;                  /* amplitude coefficient of the transverse profile */
  int n;                       /* flying focus: component count */
  double fw[OR_MAX_COMP], fk[OR_MAX_COMP], fz[OR_MAX_COMP], ft[OR_MAX_COMP];
  double fphi[OR_MAX_COMP], fzR[OR_MAX_COMP];
  double z_mid, t_mid;         /* flying focus: middle of the focal range and its time */
  double zeta;                 /* plasma: current phase factor zeta (1 in the continuum) */
  double jamp;                 /* plasma: omega_p^2 zeta / omega, J1 per unit field */
  double fdc;                  /* plasma: 1 - v_phi / v_g, weight of B's finite-duration terms */
} or_state;

/* Derive all constants from the physical description.  Returns 0, or -1 for
 * an invalid description. */
int or_prepare(const or_pulse *p, or_state *s);

/* Envelope Gamma(eta). */
double or_envelope(const or_state *s, double eta);

/* Logarithmic derivatives L1 = Gamma'/Gamma and L2 = Gamma''/Gamma of the
 * envelope at eta (the finite-duration terms of Eqs. j1 and b_corr_t).
 * Returns 0, or -1 for the sin^2 envelope (not twice differentiable at its
 * ends). */
int or_envelope_logd(const or_state *s, double eta, double *L1, double *L2);

/* Complex transverse profile u of one beam (component j for the flying focus,
 * ignored otherwise) at (x, y, z) and time t (used by the closed-form flying
 * focus only), returned as re/im. */
void or_profile(const or_state *s, int j, double x, double y, double z, double t, double *re,
                double *im);

/* Analytic E1, B1 at (x, y, z, t): EB = {Ex, Ey, Ez, Bx, By, Bz}. */
void or_fields(const or_state *s, double x, double y, double z, double t, double EB[6]);

/* Analytic current J1 (Sec. 4, Eq. j1 with Phi = 0) at (x, y, z, t):
 * J = {Jx, Jy, Jz}, zero unless omega_p > 0.  J stands for 4 pi J / c in the
 * field units, so that Ampere's law reads dE/dt = curl B - J and the linear
 * cold-plasma current obeys dJ/dt = omega_p^2 zeta E. */
void or_current(const or_state *s, double x, double y, double z, double t, double J[3]);

/* Trilinear gather of a static node-centred grid, layout [6][nz][ny][nx]
 * (x fastest), nodes at lo + i (hi - lo)/(n - 1); positions outside the box
 * are clamped to it. */
void or_grid_sample(const float *grid, int nx, int ny, int nz, const double lo[3],
                    const double hi[3], double x, double y, double z, double out[6]);

/* One relativistic Boris step of an electron (q = -1, m = 1) in E, B:
 * u is u^{n-1/2} on entry and u^{n+1/2} on exit. */
void or_boris(double u[3], const double E[3], const double B[3], double dt);

/* Push n particles for n_steps steps.  On entry x is at t0 and u at
 * t0 - dt/2; on exit x is at t0 + n_steps dt and u at t0 + (n_steps - 1/2) dt.
 * grid may be NULL.  lf_max (nullable, length n_steps) receives per step the
 * maximum over particles of |(gamma - u_z) - h0|, h0 = gamma - u_z on entry
 * (it is max-accumulated, the caller initialises it).  Returns 0. */
int or_push(const or_state *s, const float *grid, int nx, int ny, int nz, const double *glo,
            const double *ghi, int64_t n, double *x, double *y, double *z, double *ux,
            double *uy, double *uz, double t0, double dt, int64_t n_steps, double *lf_max);

/* Histogram of gamma = sqrt(((ux ux + uy uy) + uz uz) + 1) into nbins bins of
 * [lo, hi): bin = floor((gamma - lo) * (nbins / (hi - lo))), clamped to
 * [0, nbins - 1]; non-finite gamma is not counted.  Accumulates into counts. */
void or_gamma_hist(int64_t n, const double *ux, const double *uy, const double *uz, int nbins,
                   double lo, double hi, uint32_t *counts);

/* Sum of gamma over each set s of particles [off[s], off[s+1]). */
void or_set_gamma_sums(int n_sets, const int64_t *off, const double *ux, const double *uy,
                       const double *uz, double *sums);

/* Yee-staggered samples of the analytic E1, B1 on a grid (Sec. 2.1 and
 * Fig. 1: the analytic fields are set on the grid nodes every step and summed
 * with the fields the grid solver advances).  Node (i, j, k) sits at
 * lo + (i dx, j dy, k dz); inside the cell the six components sit at the
 * usual Yee offsets, in cells:
 *   Ex (1/2, 0, 0), Ey (0, 1/2, 0), Ez (0, 0, 1/2),
 *   Bx (0, 1/2, 1/2), By (1/2, 0, 1/2), Bz (1/2, 1/2, 0).
 * An unused axis has n = 1 and d = 0.  E and B are both at time t (the scheme
 * of Sec. 2.1 holds B at whole steps too).  out: [6][nz][ny][nx], x fastest. */
void or_yee_nodes(const or_state *s, int nx, int ny, int nz, const double lo[3],
                  const double d[3], double t, double *out);

/* n_steps steps of the second-order Yee scheme in vacuum for a wave along z,
 * in the three-substep form of Sec. 2.1 (the paper's x, E_y, B_z become z,
 * E_x, B_y here): E[k] = E_x at z_k, B[k] = B_y at z_{k + 1/2}, both at whole
 * time levels, r = dt / dz:
 *   B[k] -= (r/2) (E[k+1] - E[k]),  k = 0 .. nz-2
 *   E[k] -= r (B[k] - B[k-1]),       k = 1 .. nz-1
 *   B[k] -= (r/2) (E[k+1] - E[k]),  k = 0 .. nz-2
 * E[0] and B[nz-1] are never updated (fixed ends). */
void or_yee1d(int64_t nz, double *E, double *B, double dz, double dt, int64_t n_steps);

/* n_steps steps of the same line with a linear cold-plasma current J on the
 * whole nodes (J[k] at z_k and half time levels), the traditional
 * simulation that Sec. 4 compares against:
 *   B half step as above;
 *   J[k] += (dt wp2[k]) E[k],                  k = 0 .. nz-1  (J^{n+1/2})
 *   E[k] = (E[k] - r (B[k] - B[k-1])) - dt J[k],  k = 1 .. nz-1
 *   B half step with the new E.
 * wp2[k] = omega_p^2 at z_k.  With wp2 = 0 this is or_yee1d. */
void or_plasma1d(int64_t nz, double *E, double *B, double *J, const double *wp2, double dz,
                 double dt, int64_t n_steps);

/* n_steps steps of the line in the split form of Sec. 4 (Eqs. E_1_j, E_2_j):
 * E2, B2 are the internally advanced fields, J the physical plasma current,
 * driven by the total field E1 + E2; the E2 update takes the source
 * J - J1 with the analytic E1 at (z_k, t_n) and J1 at (z_k, t_n + dt/2),
 * t_n = t0 + n dt, z_k = z0 + k dz:
 *   B2 half step;
 *   J[k] += (dt wp2[k]) (E1 + E2[k]);
 *   E2[k] = (E2[k] - r (B2[k] - B2[k-1])) - dt (J[k] - J1);
 *   B2 half step.
 * The line carries E_x and B_y: the pulse must be linearly polarised along
 * x.  Returns 0, or -1 for another polarisation. */
int or_apt1d(const or_state *s, int64_t nz, double *E2, double *B2, double *J, const double *wp2,
             double z0, double dz, double t0, double dt, int64_t n_steps);

#ifdef __cplusplus
}
#endif
#endif
