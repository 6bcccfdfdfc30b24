/*
 * oracle.c -- plain FP64 CPU oracle (test infrastructure only; see oracle.h).
 *
 * Every function follows the paper (arXiv:2307.04843) or, where the paper is
 * silent, the textbook definition named beside it.  No blocking, fusion or
 * reordering: one particle at a time, one step at a time, one formula at a
 * time, so that each line can be checked against the source by eye.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stddef.h>

static const double OR_PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- helpers */

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

static double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= (double)i;
  return r;
}

/* Generalised Laguerre polynomial, explicit textbook sum
 *   L_p^a(s) = sum_{i=0}^{p} (-1)^i C(p + a, p - i) s^i / i!   */
static double laguerre(int p, int a, double s) {
  double sum = 0.0;
  for (int i = 0; i <= p; ++i) {
    double term = binom(p + a, p - i) * pow(s, (double)i) / factorial(i);
    sum += (i % 2 == 0) ? term : -term;
  }
  return sum;
}

/* Radial shape of LG_pl in the focal plane as a function of s = 2 r^2 / w0^2:
 * s^{|l|/2} |L_p^{|l|}(s)| e^{-s/2}. */
static double lg_focal_shape(int p, int al, double s) {
  return pow(s, 0.5 * al) * fabs(laguerre(p, al, s)) * exp(-0.5 * s);
}

/* max over s >= 0 of lg_focal_shape: dense sampling, then golden-section
 * refinement around the best sample. */
static double lg_focal_max(int p, int al) {
  const int ns = 20000;
  const double smax = 8.0 * (p + al + 1) + 40.0;
  double best = -1.0, sbest = 0.0;
  for (int i = 0; i <= ns; ++i) {
    double s = smax * (double)i / ns;
    double f = lg_focal_shape(p, al, s);
    if (f > best) { best = f; sbest = s; }
  }
  double a = sbest - smax / ns, b = sbest + smax / ns;
  if (a < 0.0) a = 0.0;
  const double g = 0.5 * (sqrt(5.0) - 1.0);
  for (int it = 0; it < 200; ++it) {
    double c = b - g * (b - a), d = a + g * (b - a);
    if (lg_focal_shape(p, al, c) > lg_focal_shape(p, al, d)) b = d; else a = c;
  }
  double f = lg_focal_shape(p, al, 0.5 * (a + b));
  return f > best ? f : best;
}

static void polarisation(int pol, double complex *px, double complex *py) {
  switch (pol) {
    case OR_LIN_Y: *px = 0.0; *py = 1.0; break;
    case OR_CIRC_P: *px = 1.0; *py = -I; break;
    case OR_CIRC_M: *px = 1.0; *py = I; break;
    default: *px = 1.0; *py = 0.0; break;
  }
}

/* ------------------------------------------------------------------ setup */

/* Plane wave in a linear cold plasma (Sec. 4).  With the second-order Yee
 * scheme and the current advanced by the leapfrog dJ/dt = omega_p^2 E at the
 * half steps, the current lags the continuum one by the factor
 * zeta = (omega dt/2) / sin(omega dt/2); k then follows from Eq. dispersion_j,
 *   sin^2(omega dt/2) - (omega_p^2/omega^2)(omega dt/2) sin(omega dt/2) zeta
 *     = (c dt/dx)^2 sin^2(k dx/2),
 * and B0/E0 from Eq. e_amp_j.  With this zeta the plasma term equals
 * (omega_p dt/2)^2 whatever omega is, so v_g = d omega/dk is the ratio of the
 * two sides' derivatives,
 *   v_g = (c dt/dx)^2 sin(k dx/2) cos(k dx/2) dx / (sin(omega dt/2) cos(omega dt/2) dt).
 * Without the Yee flag: the continuum, omega^2 = omega_p^2 + c^2 k^2,
 * zeta = 1, v_g = c^2 k / omega, B0/E0 = c k / omega. */
static int or_prepare_plasma(const or_pulse *p, or_state *s) {
  const double w = p->omega, wp = p->omega_p;
  if (!(wp > 0.0) || p->kind != OR_PLANE || p->env == OR_ENV_SIN2) return -1;
  if (p->yee) {
    const double h = 0.5 * w * p->yee_dt;
    if (!(h < 0.5 * OR_PI)) return -1;
    const double sw = sin(h), cw = cos(h);
    const double r = p->yee_dt / p->yee_dx;
    s->zeta = h / sw;
    const double lhs = sw * sw - (wp * wp) / (w * w) * h * sw * s->zeta;
    const double sk2 = lhs / (r * r);
    if (!(sk2 > 0.0 && sk2 < 1.0)) return -1;
    const double sk = sqrt(sk2), ck = sqrt(1.0 - sk2);
    s->k = (2.0 / p->yee_dx) * asin(sk);
    s->vg = r * r * sk * ck * p->yee_dx / (sw * cw * p->yee_dt);
    s->bratio = cw * sqrt(1.0 - (wp * wp) / (w * w) * s->zeta * h / sw);
  } else {
    if (!(wp < w)) return -1;
    s->zeta = 1.0;
    s->k = sqrt(w * w - wp * wp);
    s->vg = s->k / w;
    s->bratio = s->k / w;
  }
  s->vphi = w / s->k;
  s->jamp = wp * wp * s->zeta / w;
  s->fdc = 1.0 - s->vphi / s->vg;
  return 0;
}

int or_prepare(const or_pulse *p, or_state *s) {
  s->p = *p;
  if (!(p->omega > 0.0)) return -1;
  if (p->kind < OR_PLANE || p->kind > OR_FLYING_CF) return -1;
  /* Phase velocity, group velocity and B0/E0: vacuum unless the second-order
   * Yee expressions are requested (Eqs. vphi, vg, e_amp, Sec. 2.1). */
  s->vphi = 1.0;
  s->vg = 1.0;
  s->bratio = 1.0;
  s->zeta = 1.0;
  s->jamp = 0.0;
  s->fdc = 0.0;
  if (p->yee) {
    if (!(p->yee_dx > 0.0) || !(p->yee_dt > 0.0) || p->kind == OR_FLYING) return -1;
    double cr = p->yee_dt / p->yee_dx;
    double wdx = p->omega * p->yee_dx;
    s->vphi = 1.0 - (1.0 / 24.0) * (1.0 - cr * cr) * wdx * wdx;
    s->vg = 1.0 - (1.0 / 8.0) * (1.0 - cr * cr) * wdx * wdx;
    s->bratio = 1.0 - (p->omega * p->yee_dt) * (p->omega * p->yee_dt) / 8.0;
  }
  s->k = p->omega / s->vphi;
  if (p->omega_p != 0.0 && or_prepare_plasma(p, s) != 0) return -1;
  s->zR = 0.5 * s->k * p->w0 * p->w0;
  s->amp = p->a0;
  s->n = 0;
  if (p->kind != OR_PLANE) {
    if (!(p->w0 > 0.0)) return -1;
  }
  if (p->kind == OR_FLYING_CF && !(p->beta_f < 1.0)) return -1;
  if (p->kind == OR_LG) {
    if (p->lg_p < 0) return -1;
    int al = p->lg_l < 0 ? -p->lg_l : p->lg_l;
    /* a0 is the peak of |u| in the focal plane. */
    s->amp = p->a0 / lg_focal_max(p->lg_p, al);
  }
  if (p->kind == OR_FLYING) {
    int n = p->n_comp;
    if (n < 2 || n > OR_MAX_COMP || !(p->beta_f != 0.0)) return -1;
    s->n = n;
    /* Spectral components: equally spaced frequencies over
     * omega (1 +- bw_frac); component j focuses at z_j, equally spaced over
     * [z_a, z_a + L], and reaches it at t_j = t_a + (z_j - z_a) / v_f, so that
     * the focus moves at v_f (Sec. 3.3).  The spectral phase is the trapezoid
     * integral of the group delay tau_j = t_j - z_j over frequency. */
    for (int j = 0; j < n; ++j) {
      double fj = (double)j / (double)(n - 1);
      s->fw[j] = p->omega * (1.0 - p->bw_frac + 2.0 * p->bw_frac * fj);
      s->fk[j] = s->fw[j];
      s->fz[j] = p->z_focus + p->ff_length * fj;
      s->ft[j] = p->t_focus + (s->fz[j] - p->z_focus) / p->beta_f;
      s->fzR[j] = 0.5 * s->fk[j] * p->w0 * p->w0;
    }
    s->fphi[0] = 0.0;
    for (int j = 1; j < n; ++j) {
      double tau_j = s->ft[j] - s->fz[j];
      double tau_m = s->ft[j - 1] - s->fz[j - 1];
      s->fphi[j] = s->fphi[j - 1] + 0.5 * (tau_j + tau_m) * (s->fw[j] - s->fw[j - 1]);
    }
    s->z_mid = p->z_focus + 0.5 * p->ff_length;
    s->t_mid = p->t_focus + 0.5 * p->ff_length / p->beta_f;
    /* Common amplitude: a0 over the largest on-axis envelope |S| at t_mid,
     * S = sum_j u_j e^{i psi_j} with unit-amplitude components, sampled at
     * 2049 equally spaced z over [z_mid - L/4, z_mid + L/4]. */
    s->amp = 1.0;
    double best = 0.0;
    const int M = 2048;
    for (int i = 0; i <= M; ++i) {
      double zi = s->z_mid - 0.25 * p->ff_length + 0.5 * p->ff_length * (double)i / (double)M;
      double complex S = 0.0;
      for (int j = 0; j < n; ++j) {
        double ur, ui;
        or_profile(s, j, 0.0, 0.0, zi, 0.0, &ur, &ui);
        double psi = s->fw[j] * s->t_mid - s->fk[j] * zi - s->fphi[j];
        S += (ur + I * ui) * cexp(I * psi);
      }
      if (cabs(S) > best) best = cabs(S);
    }
    if (!(best > 0.0)) return -1;
    s->amp = p->a0 / best;
  }
  return 0;
}

/* ---------------------------------------------------------------- envelope */

double or_envelope(const or_state *s, double eta) {
  const or_pulse *p = &s->p;
  switch (p->env) {
    case OR_ENV_SIN2: {
      /* N-cycle sin^2 envelope: total support T = 2 pi N / omega. */
      double T = 2.0 * OR_PI * p->env_len / p->omega;
      if (fabs(eta) > 0.5 * T) return 0.0;
      double c = cos(OR_PI * eta / T);
      return c * c;
    }
    case OR_ENV_GAUSS:
      /* Gaussian whose intensity (Gamma^2) has full width at half maximum T. */
      return exp(-2.0 * log(2.0) * eta * eta / (p->env_len * p->env_len));
    case OR_ENV_SGAUSS:
      /* super-Gaussian of order g (Sec. 2.3): falls to 1/e at |eta| = tau. */
      return exp(-pow(fabs(eta / p->env_len), 2.0 * p->sg_order));
    default:
      return 1.0;
  }
}

/* Logarithmic derivatives of the envelope: ln Gamma is -2 ln2 eta^2 / T^2
 * (Gaussian) or -(eta/tau)^(2g) (super-Gaussian), so
 *   L1 = (ln Gamma)',  L2 = Gamma''/Gamma = L1^2 + (ln Gamma)''. */
int or_envelope_logd(const or_state *s, double eta, double *L1, double *L2) {
  const or_pulse *p = &s->p;
  switch (p->env) {
    case OR_ENV_GAUSS: {
      double a = 2.0 * log(2.0) / (p->env_len * p->env_len);
      *L1 = -2.0 * a * eta;
      *L2 = (*L1) * (*L1) - 2.0 * a;
      return 0;
    }
    case OR_ENV_SGAUSS: {
      double g = (double)p->sg_order, tau = p->env_len, u = eta / tau;
      *L1 = -2.0 * g * pow(u, 2.0 * g - 1.0) / tau;
      *L2 = (*L1) * (*L1) - 2.0 * g * (2.0 * g - 1.0) * pow(u, 2.0 * g - 2.0) / (tau * tau);
      return 0;
    }
    case OR_ENV_SIN2:
      *L1 = 0.0;
      *L2 = 0.0;
      return -1;
    default:
      *L1 = 0.0;
      *L2 = 0.0;
      return 0;
  }
}

/* ----------------------------------------------------------------- beams */

/* Paraxial beam in the +z, e^{i(omega t - k z)} convention: Eq. paraxial with
 * D = 3 and x_f - x -> z_f - z, i.e. w = w0 sqrt(1 + zeta^2),
 * 1/R = (z - z_f) / ((z - z_f)^2 + z_R^2), Gouy phase atan(zeta),
 *   u = A (w0/w) e^{-r^2/w^2} e^{-i k r^2 / (2R)} e^{+i atan zeta}
 * and for LG_pl (textbook) the extra factor
 *   (sqrt(2) r / w)^{|l|} L_p^{|l|}(2 r^2 / w^2) e^{i (2p + |l|) atan zeta} e^{i l theta}. */
void or_profile(const or_state *s, int j, double x, double y, double z, double t, double *re,
                double *im) {
  const or_pulse *p = &s->p;
  double zf = s->p.z_focus, zR = s->zR, k = s->k, A = s->amp;
  if (p->kind == OR_PLANE) { *re = A; *im = 0.0; return; }
  if (p->kind == OR_FLYING) { zf = s->fz[j]; zR = s->fzR[j]; k = s->fk[j]; }
  double dz = z - zf;
  if (p->kind == OR_FLYING_CF) {
    /* Sec. 3.3: Eq. paraxial with x_f - x -> xi0 - xi, xi = z - v_f t,
     * xi0 = z_f - v_f t_f, and the wavenumber of the transverse profile
     * k (1 - beta_f), so that x_R -> (1 - beta_f) x_R and the profile solves
     * the reduced flying-focus paraxial equation. */
    dz = (z - p->beta_f * t) - (p->z_focus - p->beta_f * p->t_focus);
    zR = (1.0 - p->beta_f) * s->zR;
    k = (1.0 - p->beta_f) * s->k;
  }
  double zeta = dz / zR;
  double w = p->w0 * sqrt(1.0 + zeta * zeta);
  double invR = dz / (dz * dz + zR * zR);
  double gouy = atan(zeta);
  double r2 = x * x + y * y;
  double mag = A * (p->w0 / w) * exp(-r2 / (w * w));
  double phase = -0.5 * k * r2 * invR + gouy;
  if (p->kind == OR_LG) {
    int al = p->lg_l < 0 ? -p->lg_l : p->lg_l;
    double sarg = 2.0 * r2 / (w * w);
    mag *= pow(sarg, 0.5 * al) * laguerre(p->lg_p, al, sarg);
    phase += (double)(2 * p->lg_p + al) * gouy + (double)p->lg_l * atan2(y, x);
  }
  *re = mag * cos(phase);
  *im = mag * sin(phase);
}

static double complex profile_c(const or_state *s, int j, double x, double y, double z, double t) {
  double re, im;
  or_profile(s, j, x, y, z, t, &re, &im);
  return re + I * im;
}

/* 4th-order central differences of the profile in x and y, h = 1e-3 w0. */
static void profile_grad(const or_state *s, int j, double x, double y, double z, double t,
                         double complex *dx, double complex *dy) {
  double h = 1e-3 * s->p.w0;
  *dx = (profile_c(s, j, x - 2 * h, y, z, t) - 8.0 * profile_c(s, j, x - h, y, z, t) +
         8.0 * profile_c(s, j, x + h, y, z, t) - profile_c(s, j, x + 2 * h, y, z, t)) / (12.0 * h);
  *dy = (profile_c(s, j, x, y - 2 * h, z, t) - 8.0 * profile_c(s, j, x, y - h, z, t) +
         8.0 * profile_c(s, j, x, y + h, z, t) - profile_c(s, j, x, y + 2 * h, z, t)) / (12.0 * h);
}

/* ---------------------------------------------------------------- fields */

void or_fields(const or_state *s, double x, double y, double z, double t, double EB[6]) {
  const or_pulse *p = &s->p;
  double complex px, py;
  polarisation(p->pol, &px, &py);
  double complex U = 0.0, DX = 0.0, DY = 0.0; /* transverse phasor, longitudinal phasors */
  double complex UB = 0.0;                     /* phasor of the transverse B */
  const int lon = p->longitudinal && p->kind != OR_PLANE;
  if (p->kind == OR_FLYING) {
    /* Linear superposition of the spectral components (Sec. 3.3); no
     * envelope: the chirp localises the pulse. */
    for (int j = 0; j < s->n; ++j) {
      double psi = s->fw[j] * t - s->fk[j] * z - s->fphi[j] + p->phase0;
      double complex ph = cexp(I * psi);
      U += profile_c(s, j, x, y, z, t) * ph;
      if (lon) {
        double complex gx, gy;
        profile_grad(s, j, x, y, z, t, &gx, &gy);
        /* divergence conditions: d/dz -> -i k_j */
        DX += (-I / s->fk[j]) * gx * ph;
        DY += (-I / s->fk[j]) * gy * ph;
      }
    }
    UB = U;
  } else {
    double eta = (t - p->t_focus) - (z - p->z_focus) / s->vg;
    double G = or_envelope(s, eta);
    double psi = p->omega * (t - p->t_focus) - s->k * (z - p->z_focus) + p->phase0;
    double complex ph = G * cexp(I * psi);
    U = profile_c(s, 0, x, y, z, t) * ph;
    UB = U;
    if (p->omega_p != 0.0) {
      /* Eq. b_corr_t with Phi = 0: the lowest finite-duration terms, weighted
       * by 1 - v_phi/v_g, change B's amplitude by the factor
       *   1 - c L2/omega^2 + (c L1/omega)^2 / 2
       * and shift its phase by c L1/omega (c = 1 - v_phi/v_g, L1 and L2 the
       * logarithmic derivatives of Gamma). */
      double L1, L2;
      or_envelope_logd(s, eta, &L1, &L2);
      double th = s->fdc * L1 / p->omega;
      double A = 1.0 - s->fdc * L2 / (p->omega * p->omega) + 0.5 * th * th;
      UB = profile_c(s, 0, x, y, z, t) * A * G * cexp(I * (psi + th));
    }
    if (lon) {
      double complex gx, gy;
      profile_grad(s, 0, x, y, z, t, &gx, &gy);
      DX = gx * ph;
      DY = gy * ph;
    }
  }
  /* Transverse fields: E_perp = Re[U p], B_perp = (B0/E0) z x E_perp
   * (Eqs. plane_func, plane_b; Eq. b_corr_t in a plasma). */
  EB[0] = creal(px * U);
  EB[1] = creal(py * U);
  EB[3] = s->bratio * creal(-py * UB);
  EB[4] = s->bratio * creal(px * UB);
  EB[2] = 0.0;
  EB[5] = 0.0;
  if (lon) {
    if (p->kind == OR_FLYING) {
      /* the -i/k_j factors are already inside DX, DY */
      EB[2] = creal(px * DX + py * DY);
      EB[5] = s->bratio * creal(-py * DX + px * DY);
    } else {
      /* div E = 0 with d/dz -> -i omega / v_phi; div B = 0 with d/dz -> -i omega / c
       * (Sec. 3.1, below Eq. paraxial). */
      EB[2] = creal((-I * s->vphi / p->omega) * (px * DX + py * DY));
      EB[5] = s->bratio * creal((-I / p->omega) * (-py * DX + px * DY));
    }
  }
}

/* Eq. j1 with Phi = 0: the current of the linear plasma response,
 *   J = Re[-i (omega_p^2 zeta / omega) A Gamma e^{i (psi + L1/omega)} p],
 *   A = 1 - L2/omega^2 + (L1/omega)^2 / 2,
 * the lowest finite-duration terms of the series in (i/omega)^n d^n/dt^n. */
void or_current(const or_state *s, double x, double y, double z, double t, double J[3]) {
  const or_pulse *p = &s->p;
  J[0] = J[1] = J[2] = 0.0;
  if (p->omega_p == 0.0) return;
  double complex px, py;
  polarisation(p->pol, &px, &py);
  double eta = (t - p->t_focus) - (z - p->z_focus) / s->vg;
  double G = or_envelope(s, eta);
  double psi = p->omega * (t - p->t_focus) - s->k * (z - p->z_focus) + p->phase0;
  double L1, L2;
  or_envelope_logd(s, eta, &L1, &L2);
  double th = L1 / p->omega;
  double A = 1.0 - L2 / (p->omega * p->omega) + 0.5 * th * th;
  double complex V = -I * s->jamp * profile_c(s, 0, x, y, z, t) * A * G * cexp(I * (psi + th));
  J[0] = creal(px * V);
  J[1] = creal(py * V);
}

/* ------------------------------------------------------------------ grid */

void or_grid_sample(const float *grid, int nx, int ny, int nz, const double lo[3],
                    const double hi[3], double x, double y, double z, double out[6]) {
  const int n[3] = {nx, ny, nz};
  const double c[3] = {x, y, z};
  int i0[3];
  double w[3];
  for (int a = 0; a < 3; ++a) {
    double v = c[a];
    if (v < lo[a]) v = lo[a];
    if (v > hi[a]) v = hi[a];
    double d = (hi[a] - lo[a]) / (double)(n[a] - 1);
    double f = (v - lo[a]) / d;
    int i = (int)floor(f);
    if (i > n[a] - 2) i = n[a] - 2;
    if (i < 0) i = 0;
    i0[a] = i;
    w[a] = f - (double)i;
  }
  const size_t plane = (size_t)nx * ny, vol = plane * nz;
  for (int comp = 0; comp < 6; ++comp) {
    const float *g = grid + comp * vol;
    double acc = 0.0;
    for (int cz = 0; cz < 2; ++cz)
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
          double wt = (cx ? w[0] : 1.0 - w[0]) * (cy ? w[1] : 1.0 - w[1]) *
                      (cz ? w[2] : 1.0 - w[2]);
          size_t idx = (size_t)(i0[2] + cz) * plane + (size_t)(i0[1] + cy) * nx + (i0[0] + cx);
          acc += wt * (double)g[idx];
        }
    out[comp] = acc;
  }
}

/* ----------------------------------------------------------------- Boris */

/* Relativistic Boris rotation (Boris 1970) for charge -1, mass 1:
 * half electric kick, magnetic rotation, half electric kick. */
void or_boris(double u[3], const double E[3], const double B[3], double dt) {
  const double h = -0.5 * dt; /* q dt / (2 m) */
  double um[3], up[3], tau[3], sv[3];
  for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  for (int a = 0; a < 3; ++a) tau[a] = h * B[a] / gm;
  double t2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
  for (int a = 0; a < 3; ++a) sv[a] = 2.0 * tau[a] / (1.0 + t2);
  double uprime[3] = {um[0] + (um[1] * tau[2] - um[2] * tau[1]),
                      um[1] + (um[2] * tau[0] - um[0] * tau[2]),
                      um[2] + (um[0] * tau[1] - um[1] * tau[0])};
  up[0] = um[0] + (uprime[1] * sv[2] - uprime[2] * sv[1]);
  up[1] = um[1] + (uprime[2] * sv[0] - uprime[0] * sv[2]);
  up[2] = um[2] + (uprime[0] * sv[1] - uprime[1] * sv[0]);
  for (int a = 0; a < 3; ++a) u[a] = up[a] + h * E[a];
}

/* ------------------------------------------------------------------ push */

int or_push(const or_state *s, const float *grid, int nx, int ny, int nz, const double *glo,
            const double *ghi, int64_t n, double *x, double *y, double *z, double *ux,
            double *uy, double *uz, double t0, double dt, int64_t n_steps, double *lf_max) {
  for (int64_t i = 0; i < n; ++i) {
    double pos[3] = {x[i], y[i], z[i]};
    double u[3] = {ux[i], uy[i], uz[i]};
    double h0 = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) - u[2];
    for (int64_t st = 0; st < n_steps; ++st) {
      double t = t0 + (double)st * dt; /* t_n = t0 + n dt, not accumulated */
      double EB[6];
      or_fields(s, pos[0], pos[1], pos[2], t, EB);
      if (grid) {
        /* E = E1 + E2, B = B1 + B2 (Eqs. E_1, E_2): analytic plus gathered */
        double g6[6];
        or_grid_sample(grid, nx, ny, nz, glo, ghi, pos[0], pos[1], pos[2], g6);
        for (int c = 0; c < 6; ++c) EB[c] += g6[c];
      }
      or_boris(u, EB, EB + 3, dt);
      double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      /* 1D-3V (Sec. 3.2): only z moves; the momentum keeps all three components */
      for (int a = s->p.one_d ? 2 : 0; a < 3; ++a) pos[a] += dt * u[a] / g;
      if (lf_max) {
        double dev = fabs((g - u[2]) - h0);
        if (dev > lf_max[st]) lf_max[st] = dev;
      }
    }
    x[i] = pos[0]; y[i] = pos[1]; z[i] = pos[2];
    ux[i] = u[0]; uy[i] = u[1]; uz[i] = u[2];
  }
  return 0;
}

/* ----------------------------------------------------------- diagnostics */

void or_gamma_hist(int64_t n, const double *ux, const double *uy, const double *uz, int nbins,
                   double lo, double hi, uint32_t *counts) {
  double scale = (double)nbins / (hi - lo);
  for (int64_t i = 0; i < n; ++i) {
    double g = sqrt(((ux[i] * ux[i] + uy[i] * uy[i]) + uz[i] * uz[i]) + 1.0);
    if (!isfinite(g)) continue;
    double f = floor((g - lo) * scale);
    int64_t b = f < 0.0 ? 0 : (f > (double)(nbins - 1) ? nbins - 1 : (int64_t)f);
    counts[b] += 1;
  }
}

void or_set_gamma_sums(int n_sets, const int64_t *off, const double *ux, const double *uy,
                       const double *uz, double *sums) {
  for (int st = 0; st < n_sets; ++st) {
    double acc = 0.0;
    for (int64_t i = off[st]; i < off[st + 1]; ++i)
      acc += sqrt(1.0 + ux[i] * ux[i] + uy[i] * uy[i] + uz[i] * uz[i]);
    sums[st] = acc;
  }
}

/* ------------------------------------------------------------ Yee grid */

/* Offsets of Ex, Ey, Ez, Bx, By, Bz inside the Yee cell (Yee 1966), in cells. */
static const double yee_offset[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},
};

void or_yee_nodes(const or_state *s, int nx, int ny, int nz, const double lo[3],
                  const double d[3], double t, double *out) {
  const int64_t plane = (int64_t)nx * ny * nz;
  for (int c = 0; c < 6; ++c) {
    for (int k = 0; k < nz; ++k) {
      for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
          double x = lo[0] + (i + yee_offset[c][0]) * d[0];
          double y = lo[1] + (j + yee_offset[c][1]) * d[1];
          double z = lo[2] + (k + yee_offset[c][2]) * d[2];
          double EB[6];
          or_fields(s, x, y, z, t, EB);
          out[c * plane + ((int64_t)k * ny + j) * nx + i] = EB[c];
        }
      }
    }
  }
}

void or_yee1d(int64_t nz, double *E, double *B, double dz, double dt, int64_t n_steps) {
  const double r = dt / dz;
  for (int64_t n = 0; n < n_steps; ++n) {
    for (int64_t k = 0; k + 1 < nz; ++k) B[k] -= 0.5 * r * (E[k + 1] - E[k]);
    for (int64_t k = 1; k < nz; ++k) E[k] -= r * (B[k] - B[k - 1]);
    for (int64_t k = 0; k + 1 < nz; ++k) B[k] -= 0.5 * r * (E[k + 1] - E[k]);
  }
}

void or_plasma1d(int64_t nz, double *E, double *B, double *J, const double *wp2, double dz,
                 double dt, int64_t n_steps) {
  const double r = dt / dz;
  for (int64_t n = 0; n < n_steps; ++n) {
    for (int64_t k = 0; k + 1 < nz; ++k) B[k] -= 0.5 * r * (E[k + 1] - E[k]);
    for (int64_t k = 0; k < nz; ++k) J[k] += dt * wp2[k] * E[k];
    for (int64_t k = 1; k < nz; ++k) E[k] = (E[k] - r * (B[k] - B[k - 1])) - dt * J[k];
    for (int64_t k = 0; k + 1 < nz; ++k) B[k] -= 0.5 * r * (E[k + 1] - E[k]);
  }
}

int or_apt1d(const or_state *s, int64_t nz, double *E2, double *B2, double *J, const double *wp2,
             double z0, double dz, double t0, double dt, int64_t n_steps) {
  if (s->p.pol != OR_LIN_X) return -1;
  const double r = dt / dz;
  double EB[6], J1[3];
  for (int64_t n = 0; n < n_steps; ++n) {
    const double t = t0 + (double)n * dt;
    for (int64_t k = 0; k + 1 < nz; ++k) B2[k] -= 0.5 * r * (E2[k + 1] - E2[k]);
    for (int64_t k = 0; k < nz; ++k) {
      or_fields(s, 0.0, 0.0, z0 + (double)k * dz, t, EB);
      J[k] += dt * wp2[k] * (EB[0] + E2[k]);
    }
    for (int64_t k = 1; k < nz; ++k) {
      or_current(s, 0.0, 0.0, z0 + (double)k * dz, t + 0.5 * dt, J1);
      E2[k] = (E2[k] - r * (B2[k] - B2[k - 1])) - dt * (J[k] - J1[0]);
    }
    for (int64_t k = 0; k + 1 < nz; ++k) B2[k] -= 0.5 * r * (E2[k + 1] - E2[k]);
  }
  return 0;
}
