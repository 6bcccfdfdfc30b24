// ap_api.cu -- the C ABI of include/ap.h: argument checks, pulse setup (row
// a1, all derived constants in FP64 on the host), buffer management of the
// handle, launches, graph capture and the device status word.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "ap_internal.h"

using apt::Pulse;

struct ap_handle_s {
  int device = 0;
  int sm_count = 1;
  int n_sets = 0;
  int uniform_kind = -1;  // kind shared by every set, else -1
  std::vector<ap_pulse_desc> descs;
  std::vector<Pulse<double>> pd;
  std::vector<Pulse<float>> pf;
  Pulse<double> *d_pd = nullptr;
  Pulse<float> *d_pf = nullptr;
  int *d_status = nullptr;
  apt::LaunchShape shape{0, 0, 0, 0, 0};
};

struct ap_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr double kPi = 3.14159265358979323846;

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

// Coefficients c_i of L_p^a(s) = sum_i c_i s^i.
void laguerre_coeffs(int p, int a, double *c) {
  double fact = 1.0;
  for (int i = 0; i <= p; ++i) {
    if (i > 0) fact *= (double)i;
    double v = binom(p + a, p - i) / fact;
    c[i] = (i & 1) ? -v : v;
  }
}

double poly(const double *c, int p, double s) {
  double r = c[p];
  for (int i = p - 1; i >= 0; --i) r = r * s + c[i];
  return r;
}

// LG focal-plane radial shape f(s) = s^{a/2} |L(s)| e^{-s/2} and its maximum:
// coarse scan, then bisection on the sign of f'(s) between the neighbours of
// the best sample (f' = e^{-s/2} s^{a/2 - 1} [ (a/2) L + s L' - s L / 2 ]).
double lg_peak(int p, int a) {
  double c[apt::kLgMaxP + 1], dc[apt::kLgMaxP + 1];
  laguerre_coeffs(p, a, c);
  for (int i = 0; i < p; ++i) dc[i] = (double)(i + 1) * c[i + 1];
  auto f = [&](double s) { return std::pow(s, 0.5 * a) * std::fabs(poly(c, p, s)) * std::exp(-0.5 * s); };
  auto g = [&](double s) {  // sign-carrying part of f'(s) times sign(L)
    double L = poly(c, p, s), dL = p > 0 ? poly(dc, p - 1, s) : 0.0;
    double v = 0.5 * a * L + s * dL - 0.5 * s * L;
    return L >= 0.0 ? v : -v;
  };
  const int ns = 4096;
  const double smax = 6.0 * (p + a + 2) + 30.0;
  int kb = 0;
  double fb = f(0.0);
  for (int k = 1; k <= ns; ++k) {
    double v = f(smax * k / ns);
    if (v > fb) { fb = v; kb = k; }
  }
  if (kb == 0) return fb;  // maximum on the axis (a = 0)
  double lo = smax * (kb - 1) / ns, hi = smax * (kb + 1) / ns;
  double s_best = smax * kb / ns;
  // f' > 0 left of the peak, < 0 right of it
  if (g(lo) > 0.0 && g(hi) < 0.0) {
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (g(mid) > 0.0) lo = mid; else hi = mid;
    }
    s_best = 0.5 * (lo + hi);
  }
  double v = f(s_best);
  return v > fb ? v : fb;
}

// Plane wave in a linear cold plasma (Sec. 4): wavenumber k, group velocity,
// B0/E0 and the current's phase factor zeta.  With AP_F_YEE_DISP the Yee
// relation of Eq. dispersion_j for a current advanced by the leapfrog
// dJ/dt = omega_p^2 E at half steps, whose zeta = h/sin h (h = omega dt/2)
// turns the plasma term into q^2, q = omega_p dt/2:
//   sin^2 h - q^2 = (dt/dx)^2 sin^2(k dx/2),
// v_g = d omega/dk from the two sides' derivatives, and Eq. e_amp_j
// B0/E0 = cos h sqrt(1 - q^2/sin^2 h).  Otherwise the continuum:
// omega^2 = omega_p^2 + k^2, v_g = k/omega, B0/E0 = k/omega, zeta = 1.
// False when no real k exists (below the cut-off, or beyond the grid's
// largest wavenumber).
bool plasma_dispersion(const ap_pulse_desc &d, double &k, double &vg, double &br, double &zeta) {
  const double w = d.omega, wp = d.omega_p;
  if (d.flags & AP_F_YEE_DISP) {
    const double h = 0.5 * w * d.yee_dt;
    if (!(h < 0.5 * kPi)) return false;
    const double sh = std::sin(h), ch = std::cos(h), r = d.yee_dt / d.yee_dx;
    const double q = 0.5 * wp * d.yee_dt;
    const double s2 = (sh * sh - q * q) / (r * r);  // sin^2(k dx/2)
    if (!(s2 > 0.0 && s2 < 1.0)) return false;
    const double sk = std::sqrt(s2), ck = std::sqrt(1.0 - s2);
    zeta = h / sh;
    k = 2.0 * std::asin(sk) / d.yee_dx;
    vg = r * r * sk * ck * d.yee_dx / (sh * ch * d.yee_dt);
    br = ch * std::sqrt(1.0 - (q * q) / (sh * sh));
  } else {
    if (!(wp < w)) return false;
    zeta = 1.0;
    k = std::sqrt((w - wp) * (w + wp));
    vg = k / w;
    br = k / w;
  }
  return true;
}

int check_desc(const ap_pulse_desc &d) {
  if (d.kind < AP_PLANE || d.kind > AP_FLYING_CF) return AP_ERR_ARG;
  if (d.kind == AP_FLYING_CF && !(d.beta_f < 1.0 && std::isfinite(d.beta_f))) return AP_ERR_ARG;
  if (d.pol < AP_LIN_X || d.pol > AP_CIRC_M) return AP_ERR_ARG;
  if (!(d.omega > 0.0) || !std::isfinite(d.a0) || !std::isfinite(d.phase0)) return AP_ERR_ARG;
  if (!std::isfinite(d.z_focus) || !std::isfinite(d.t_focus)) return AP_ERR_ARG;
  if (d.kind != AP_FLYING_SUM) {
    if (d.env < AP_ENV_SIN2 || d.env > AP_ENV_CW) return AP_ERR_ARG;
    if (d.env != AP_ENV_CW && !(d.env_len > 0.0)) return AP_ERR_ARG;
    if (d.env == AP_ENV_SGAUSS && (d.sg_order < 1 || d.sg_order > 16)) return AP_ERR_ARG;
  }
  if (d.kind != AP_PLANE && !(d.w0 > 0.0)) return AP_ERR_ARG;
  if (d.kind == AP_LG) {
    if (d.lg_p < 0 || d.lg_p > apt::kLgMaxP) return AP_ERR_ARG;
    if (d.lg_l < -apt::kLgMaxL || d.lg_l > apt::kLgMaxL) return AP_ERR_ARG;
  }
  if (d.kind == AP_FLYING_SUM) {
    if (d.n_comp < 2 || d.n_comp > AP_MAX_COMP) return AP_ERR_ARG;
    if (!(d.beta_f != 0.0) || !std::isfinite(d.beta_f)) return AP_ERR_ARG;
    if (!(d.bw_frac >= 0.0 && d.bw_frac < 1.0) || !(d.ff_length > 0.0)) return AP_ERR_ARG;
    if (d.flags & AP_F_YEE_DISP) return AP_ERR_UNSUPPORTED;
  }
  if (d.flags & AP_F_YEE_DISP) {
    if (!(d.yee_dx > 0.0) || !(d.yee_dt > 0.0) || !(d.yee_dt < d.yee_dx)) return AP_ERR_ARG;
  }
  if (d.flags & ~(AP_F_LONGITUDINAL | AP_F_YEE_DISP | AP_F_1D3V)) return AP_ERR_ARG;
  if (!(d.omega_p >= 0.0) || !std::isfinite(d.omega_p)) return AP_ERR_ARG;
  if (d.omega_p > 0.0) {
    if (d.kind != AP_PLANE) return AP_ERR_ARG;
    if (d.env != AP_ENV_GAUSS && d.env != AP_ENV_SGAUSS && d.env != AP_ENV_CW) return AP_ERR_ARG;
    double k, vg, br, zeta;
    if (!plasma_dispersion(d, k, vg, br, zeta)) return AP_ERR_ARG;
  }
  return AP_OK;
}

// Derive the device description of one pulse in double.
void derive(const ap_pulse_desc &d, Pulse<double> &P, Pulse<float> &F) {
  std::memset(&P, 0, sizeof(P));
  P.kind = d.kind;
  P.pol = d.pol;
  P.env = d.kind == AP_FLYING_SUM ? AP_ENV_CW : d.env;
  P.lon = (d.flags & AP_F_LONGITUDINAL) && d.kind != AP_PLANE ? 1 : 0;
  P.sg_order = d.sg_order;
  P.yee = (d.flags & AP_F_YEE_DISP) ? 1 : 0;
  P.adv_xy = (d.flags & AP_F_1D3V) ? 0.0 : 1.0;
  // Phase velocity, group velocity and B0/E0 (Eqs. vphi, vg, e_amp, Sec. 2.1;
  // vacuum values unless requested).
  double vphi = 1.0, vg = 1.0, br = 1.0;
  if (P.yee) {
    const double cr = d.yee_dt / d.yee_dx, wdx = d.omega * d.yee_dx, wdt = d.omega * d.yee_dt;
    vphi = 1.0 - (1.0 - cr * cr) * wdx * wdx / 24.0;
    vg = 1.0 - (1.0 - cr * cr) * wdx * wdx / 8.0;
    br = 1.0 - wdt * wdt / 8.0;
  }
  double k = d.omega / vphi, zeta = 1.0;
  if (d.omega_p > 0.0) {
    plasma_dispersion(d, k, vg, br, zeta);
    vphi = d.omega / k;
    P.plasma = 1;
    P.fdc = 1.0 - vphi / vg;
    P.jamp = d.omega_p * d.omega_p * zeta / d.omega;
  }
  P.inv_w = 1.0 / d.omega;
  if (d.env == AP_ENV_GAUSS) {  // ln Gamma = -2 ln2 eta^2 / T^2
    P.lg_c1 = 4.0 * std::log(2.0) / (d.env_len * d.env_len);
    P.lg_c2 = P.lg_c1;
  } else if (d.env == AP_ENV_SGAUSS) {  // ln Gamma = -(eta/tau)^(2g)
    const double g2 = 2.0 * d.sg_order;
    P.lg_c1 = g2 / d.env_len;
    P.lg_c2 = g2 * (g2 - 1.0) / (d.env_len * d.env_len);
  }
  P.omega = d.omega;
  P.k = k;
  P.t_f = d.t_focus;
  P.z_f = d.z_focus;
  P.phase0 = d.phase0;
  P.inv_vg = 1.0 / vg;
  P.bratio = br;
  P.lonE = vphi / d.omega;
  P.lonB = 1.0 / d.omega;
  P.amp = d.a0;
  P.a0 = d.a0;
  P.amp_unit = 1.0;
  P.inv_w0 = d.kind != AP_PLANE ? 1.0 / d.w0 : 0.0;
  if (d.kind != AP_PLANE) {
    P.inv_w0sq = 1.0 / (d.w0 * d.w0);
    P.inv_zR = 1.0 / (0.5 * k * d.w0 * d.w0);
  }
  if (d.kind == AP_FLYING_CF) {
    // Sec. 3.3: x_R -> (1 - beta_f) x_R for the moving focus
    P.beta_f = d.beta_f;
    P.inv_1mb = 1.0 / (1.0 - d.beta_f);
    P.inv_zR *= P.inv_1mb;
  }
  switch (P.env) {
    case AP_ENV_SIN2: {
      const double T = 2.0 * kPi * d.env_len / d.omega;
      P.env_a = kPi / T;
      P.env_b = 0.5 * T;
      break;
    }
    case AP_ENV_GAUSS:  // exp(-2 ln2 eta^2/T^2) = 2^(-2 eta^2 / T^2)
      P.env_a = 2.0 / (d.env_len * d.env_len);
      break;
    case AP_ENV_SGAUSS:
      P.env_a = 1.0 / d.env_len;
      P.env_b = 1.4426950408889634;
      break;
    default:
      break;
  }
  switch (d.pol) {
    case AP_LIN_Y: P.py_re = 1.0; break;
    case AP_CIRC_P: P.px_re = 1.0; P.py_im = -1.0; break;
    case AP_CIRC_M: P.px_re = 1.0; P.py_im = 1.0; break;
    default: P.px_re = 1.0; break;
  }
  if (d.kind == AP_LG) {
    const int a = d.lg_l < 0 ? -d.lg_l : d.lg_l;
    P.lg_p = d.lg_p;
    P.lg_al = a;
    P.lg_alf = (double)a;
    P.lg_sgn = d.lg_l < 0 ? -1 : 1;
    for (int k = 0; k < apt::kLgMaxP; ++k) {
      const double k1 = (double)(k + 1);
      for (int r = 0; r < 2; ++r) {
        const double aa = (double)(a + r);
        P.lg_r[3 * r + 0][k] = (2.0 * k + 1.0 + aa) / k1;
        P.lg_r[3 * r + 1][k] = 1.0 / k1;
        P.lg_r[3 * r + 2][k] = ((double)k + aa) / k1;
      }
    }
    P.lg_pref = std::pow(std::sqrt(2.0) / d.w0, (double)a);
    P.amp_unit = 1.0 / lg_peak(d.lg_p, a);
    P.amp = d.a0 * P.amp_unit;
  }
  if (d.kind == AP_FLYING_SUM) {
    // Spectral components (Sec. 3.3, linear superposition): omega_j spread
    // uniformly over omega (1 +- bw), foci z_j uniformly over [z_a, z_a + L]
    // reached at t_j = t_a + (z_j - z_a)/v_f; spectral phase Phi_j from the
    // trapezoid rule on the group delay tau_j = t_j - z_j.
    const int n = d.n_comp;
    std::vector<double> w(n), zj(n), tau(n), Phi(n), zR(n);
    for (int j = 0; j < n; ++j) {
      const double fj = (double)j / (double)(n - 1);
      w[j] = d.omega * (1.0 - d.bw_frac + 2.0 * d.bw_frac * fj);
      zj[j] = d.z_focus + d.ff_length * fj;
      tau[j] = d.t_focus + (zj[j] - d.z_focus) / d.beta_f - zj[j];
      zR[j] = 0.5 * w[j] * d.w0 * d.w0;
    }
    Phi[0] = 0.0;
    for (int j = 1; j < n; ++j) Phi[j] = Phi[j - 1] + 0.5 * (tau[j] + tau[j - 1]) * (w[j] - w[j - 1]);
    // normalisation: largest on-axis envelope at t_mid over 2049 z samples in
    // [z_mid - L/4, z_mid + L/4], unit components; on axis u_j = q_j.
    const double z_mid = d.z_focus + 0.5 * d.ff_length;
    const double t_mid = d.t_focus + 0.5 * d.ff_length / d.beta_f;
    double best = 0.0;
    for (int i = 0; i <= 2048; ++i) {
      const double z = z_mid - 0.25 * d.ff_length + 0.5 * d.ff_length * (double)i / 2048.0;
      std::complex<double> S(0.0, 0.0);
      for (int j = 0; j < n; ++j) {
        const double zeta = (z - zj[j]) / zR[j];
        const std::complex<double> q = 1.0 / std::complex<double>(1.0, -zeta);
        const double ang = w[j] * (t_mid - z) - Phi[j];
        S += q * std::complex<double>(std::cos(ang), std::sin(ang));
      }
      best = std::max(best, std::abs(S));
    }
    const double A = d.a0 / best;
    P.amp_unit = 1.0 / best;
    P.n_comp = n;
    P.ff_w = w[0];
    P.ff_dw = (w[n - 1] - w[0]) / (double)(n - 1);
    P.lonE = 1.0;  // the 1/k_j factors sit in each component
    P.lonB = 1.0;
    for (int j = 0; j < n; ++j) {
      const double th = w[j] * d.t_focus - w[j] * d.z_focus - Phi[j] + d.phase0;
      P.comp[j].inv_zR = 1.0 / zR[j];
      P.comp[j].zoff = (zj[j] - d.z_focus) / zR[j];
      P.comp[j].inv_k = 1.0 / w[j];
      P.comp[j].c_re = A * std::cos(th);
      P.comp[j].c_im = A * std::sin(th);
    }
    P.amp = A;
  }
  // float copy
  std::memset(&F, 0, sizeof(F));
  F.kind = P.kind; F.pol = P.pol; F.env = P.env; F.lon = P.lon;
  F.lg_p = P.lg_p; F.lg_al = P.lg_al; F.lg_sgn = P.lg_sgn; F.n_comp = P.n_comp;
  F.sg_order = P.sg_order; F.yee = P.yee; F.plasma = P.plasma;
  F.fdc = (float)P.fdc; F.jamp = (float)P.jamp; F.inv_w = (float)P.inv_w;
  F.lg_c1 = (float)P.lg_c1; F.lg_c2 = (float)P.lg_c2;
  F.amp = (float)P.amp; F.inv_vg = (float)P.inv_vg; F.bratio = (float)P.bratio;
  F.lonE = (float)P.lonE; F.lonB = (float)P.lonB;
  F.inv_w0sq = (float)P.inv_w0sq; F.inv_zR = (float)P.inv_zR;
  F.env_a = (float)P.env_a; F.env_b = (float)P.env_b;
  F.px_re = (float)P.px_re; F.px_im = (float)P.px_im;
  F.py_re = (float)P.py_re; F.py_im = (float)P.py_im;
  for (int r = 0; r < 6; ++r)
    for (int k = 0; k < apt::kLgMaxP; ++k) F.lg_r[r][k] = (float)P.lg_r[r][k];
  F.lg_pref = (float)P.lg_pref;
  F.lg_alf = (float)P.lg_alf;
  F.beta_f = (float)P.beta_f;
  F.adv_xy = (float)P.adv_xy;
  F.inv_1mb = (float)P.inv_1mb;
  F.a0 = (float)P.a0;
  F.inv_w0 = (float)P.inv_w0;
  F.amp_unit = (float)P.amp_unit;
  F.omega = P.omega; F.k = P.k; F.t_f = P.t_f; F.z_f = P.z_f; F.phase0 = P.phase0;
  F.ff_w = P.ff_w; F.ff_dw = P.ff_dw;
  for (int j = 0; j < P.n_comp; ++j) {
    F.comp[j].inv_zR = (float)P.comp[j].inv_zR;
    F.comp[j].zoff = (float)P.comp[j].zoff;
    F.comp[j].inv_k = (float)P.comp[j].inv_k;
    F.comp[j].c_re = (float)P.comp[j].c_re;
    F.comp[j].c_im = (float)P.comp[j].c_im;
  }
  auto split = [](double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  split(P.k, F.k_hi, F.k_lo);
  split(P.z_f, F.zf_hi, F.zf_lo);
  split(P.ff_w, F.ffw_hi, F.ffw_lo);
  split(P.ff_dw, F.ffd_hi, F.ffd_lo);
  P.k_hi = F.k_hi; P.k_lo = F.k_lo; P.zf_hi = F.zf_hi; P.zf_lo = F.zf_lo;
  P.ffw_hi = F.ffw_hi; P.ffw_lo = F.ffw_lo; P.ffd_hi = F.ffd_hi; P.ffd_lo = F.ffd_lo;
}

int current_device_matches(const ap_handle_s *h) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return AP_ERR_CUDA;
  return dev == h->device ? AP_OK : AP_ERR_ARG;
}

int check_particles(const ap_particles *p, int precision) {
  if (!p || p->n < 0) return AP_ERR_ARG;
  if (precision < AP_FP64 || precision > AP_FP32_PHASEFF) return AP_ERR_ARG;
  if (p->n == 0) return AP_OK;
  const void *ptrs[6] = {p->x, p->y, p->z, p->ux, p->uy, p->uz};
  for (const void *q : ptrs) {
    if (!q) return AP_ERR_ARG;
    if (!aligned16(q)) return AP_ERR_ALIGN;
  }
  return AP_OK;
}

int make_grid(const ap_grid *g, apt::GridView &v) {
  std::memset(&v, 0, sizeof(v));
  if (!g) return AP_OK;
  if (g->nx < 2 || g->ny < 2 || g->nz < 2) return AP_ERR_ARG;
  const int n[3] = {g->nx, g->ny, g->nz};
  if (g->packed_layout != AP_PACK_NODES && g->packed_layout != AP_PACK_CELLS) return AP_ERR_ARG;
  const bool cells = g->packed && g->packed_layout == AP_PACK_CELLS;
  if (g->packed) {
    if (!aligned16(g->packed)) return AP_ERR_ALIGN;
    if (cells) v.cells = reinterpret_cast<const float4 *>(g->packed);
    else v.packed = reinterpret_cast<const float4 *>(g->packed);
  }
  for (int c = 0; c < 6; ++c) {
    if (!g->f[c] && !v.packed && !cells) return AP_ERR_ARG;
    if (g->f[c] && (reinterpret_cast<uintptr_t>(g->f[c]) & 3u)) return AP_ERR_ALIGN;
    v.f[c] = g->f[c];
  }
  if ((double)g->nx * g->ny * g->nz > 2147483647.0) return AP_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    if (!(g->hi[a] > g->lo[a]) || !std::isfinite(g->lo[a]) || !std::isfinite(g->hi[a]))
      return AP_ERR_ARG;
    const double inv = (double)(n[a] - 1) / (g->hi[a] - g->lo[a]);
    v.lo_d[a] = g->lo[a];
    v.inv_d_d[a] = inv;
    v.lo[a] = (float)g->lo[a];
    v.inv_d[a] = (float)inv;
    v.off_d[a] = -g->lo[a] * inv;
    v.off[a] = (float)v.off_d[a];
    v.top[a] = (float)(n[a] - 1);
    v.top2[a] = (float)(n[a] - 2);
  }
  v.nx = g->nx;
  v.ny = g->ny;
  v.nz = g->nz;
  return AP_OK;
}

int make_diag(const ap_diag *d, long long n_steps, int n_sets, apt::DiagView &v, void *stream) {
  std::memset(&v, 0, sizeof(v));
  if (!d) return AP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d->lightfront_max) {
    v.lf = d->lightfront_max;
    if (!d->accumulate && n_steps > 0 &&
        cudaMemsetAsync(v.lf, 0, (size_t)n_steps * sizeof(double), s) != cudaSuccess)
      return AP_ERR_CUDA;
  }
  if (d->gamma_hist) {
    if (d->hist_bins < 1 || d->hist_bins > 8192) return AP_ERR_ARG;
    if (!(d->hist_hi > d->hist_lo)) return AP_ERR_ARG;
    v.hist = d->gamma_hist;
    v.bins = d->hist_bins;
    v.hist_lo = d->hist_lo;
    v.hist_scale = (double)d->hist_bins / (d->hist_hi - d->hist_lo);
    if (!d->accumulate &&
        cudaMemsetAsync(v.hist, 0, (size_t)d->hist_bins * sizeof(uint32_t), s) != cudaSuccess)
      return AP_ERR_CUDA;
  }
  if (d->set_gamma_sum) {
    v.set_sum = d->set_gamma_sum;
    if (!d->accumulate &&
        cudaMemsetAsync(v.set_sum, 0, (size_t)n_sets * sizeof(double), s) != cudaSuccess)
      return AP_ERR_CUDA;
  }
  return AP_OK;
}

int default_block(const ap_handle_s *h, long long n) {
  if (h->shape.block > 0) return h->shape.block;
  long long per_sm = n / (h->sm_count > 0 ? h->sm_count : 1);
  int b = 128;
  while (b > 32 && per_sm < b) b >>= 1;
  return b;
}

int fill_push_args(ap_handle_s *h, const ap_particles *p, const ap_grid *g, double t0, double dt,
                   int64_t n_steps, int32_t precision, const ap_diag *diag, int n_sets_diag,
                   apt::PushArgs &a, void *stream) {
  int rc = check_particles(p, precision);
  if (rc != AP_OK) return rc;
  if (!std::isfinite(t0) || !std::isfinite(dt) || n_steps < 0) return AP_ERR_ARG;
  // the float-float time base counts steps in float and reduces the carrier
  // phase C_n = C_0 + n (omega dt mod 2 pi) with a magic-number rounding that
  // holds for |C_n| < 2^22 (2 pi): at most 2^23 - 1 steps per call
  if (precision == AP_FP32_PHASEFF && n_steps >= (int64_t(1) << 23)) return AP_ERR_ARG;
  std::memset(&a, 0, sizeof(a));
  a.x = p->x; a.y = p->y; a.z = p->z;
  a.ux = p->ux; a.uy = p->uy; a.uz = p->uz;
  a.n = p->n;
  a.t0 = t0;
  a.dt = dt;
  a.n_steps = n_steps;
  rc = make_grid(g, a.grid);
  if (rc != AP_OK) return rc;
  a.grid_on = g != nullptr;
  // the double push interpolates the raw corners: the coefficient copy is
  // float-rounded, so it reads the component arrays instead
  if (a.grid.cells && precision == AP_FP64) {
    rc = apt::drop_cell_layout(a.grid);
    if (rc != AP_OK) return rc;
  }
  rc = make_diag(diag, n_steps, n_sets_diag, a.diag, stream);
  if (rc != AP_OK) return rc;
  a.status = h->d_status;
  a.sm_count = h->sm_count;
  a.shape = h->shape;
  a.shape.block = default_block(h, p->n);
  return AP_OK;
}

}  // namespace

namespace apt {

int drop_cell_layout(GridView &v) {
  for (int c = 0; c < 6; ++c)
    if (!v.f[c]) return AP_ERR_ARG;
  v.cells = nullptr;
  return AP_OK;
}

// Accessors used by the adjoint translation unit.
int handle_info(ap_handle h, int *device, int *sm_count, int *n_sets, int *uniform_kind,
                const Pulse<double> **dpd, const Pulse<float> **dpf, int **status) {
  if (!h) return AP_ERR_ARG;
  int rc = current_device_matches(h);
  if (rc != AP_OK) return rc;
  *device = h->device;
  *sm_count = h->sm_count;
  *n_sets = h->n_sets;
  *uniform_kind = h->uniform_kind;
  *dpd = h->d_pd;
  *dpf = h->d_pf;
  *status = h->d_status;
  return AP_OK;
}

int handle_push_args(ap_handle h, const ap_particles *p, const ap_grid *g, double t0, double dt,
                     int64_t n_steps, int32_t precision, PushArgs *a, void *stream) {
  return fill_push_args(h, p, g, t0, dt, n_steps, precision, nullptr, 1, *a, stream);
}

int launch_push(int kind, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                const PushArgs &a, void *stream) {
  switch (kind) {
    case AP_PLANE: return launch_push_plane(precision, pd, pf, a, stream);
    case AP_GAUSS: return launch_push_gauss(precision, pd, pf, a, stream);
    case AP_LG: return launch_push_lg(precision, pd, pf, a, stream);
    case AP_FLYING_SUM: return launch_push_flying(precision, pd, pf, a, stream);
    case AP_FLYING_CF: return launch_push_flyingcf(precision, pd, pf, a, stream);
    default: return AP_ERR_ARG;
  }
}

int launch_eval(int kind, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                const EvalArgs &a, void *stream) {
  switch (kind) {
    case AP_PLANE: return launch_eval_plane(precision, pd, pf, a, stream);
    case AP_GAUSS: return launch_eval_gauss(precision, pd, pf, a, stream);
    case AP_LG: return launch_eval_lg(precision, pd, pf, a, stream);
    case AP_FLYING_SUM: return launch_eval_flying(precision, pd, pf, a, stream);
    case AP_FLYING_CF: return launch_eval_flyingcf(precision, pd, pf, a, stream);
    default: return AP_ERR_ARG;
  }
}

int launch_nodes(int kind, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                 const NodeArgs &a, void *stream) {
  switch (kind) {
    case AP_PLANE: return launch_nodes_plane(precision, pd, pf, a, stream);
    case AP_GAUSS: return launch_nodes_gauss(precision, pd, pf, a, stream);
    case AP_LG: return launch_nodes_lg(precision, pd, pf, a, stream);
    case AP_FLYING_SUM: return launch_nodes_flying(precision, pd, pf, a, stream);
    case AP_FLYING_CF: return launch_nodes_flyingcf(precision, pd, pf, a, stream);
    default: return AP_ERR_ARG;
  }
}

int launch_batch(int kind, int precision, const Pulse<double> *dpd, const Pulse<float> *dpf,
                 const BatchArgs &a, void *stream) {
  switch (kind) {
    case AP_PLANE: return launch_batch_plane(precision, dpd, dpf, a, stream);
    case AP_GAUSS: return launch_batch_gauss(precision, dpd, dpf, a, stream);
    case AP_LG: return launch_batch_lg(precision, dpd, dpf, a, stream);
    case AP_FLYING_SUM: return launch_batch_flying(precision, dpd, dpf, a, stream);
    case AP_FLYING_CF: return launch_batch_flyingcf(precision, dpd, dpf, a, stream);
    default: return AP_ERR_ARG;
  }
}

}  // namespace apt

extern "C" {

int ap_version(void) { return AP_ABI_VERSION; }

const char *ap_status_string(int status) {
  switch (status) {
    case AP_OK: return "ok";
    case AP_ERR_ARG: return "invalid argument";
    case AP_ERR_ALIGN: return "device pointer not 16-byte aligned";
    case AP_ERR_CUDA: return "CUDA runtime error";
    case AP_ERR_NONFINITE: return "non-finite particle state or field";
    case AP_ERR_TIMEOUT: return "reserved (no device-side wait exists in this library)";
    case AP_ERR_WORKSPACE: return "workspace too small";
    case AP_ERR_UNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
  }
}

int ap_init_pulse(const ap_pulse_desc *descs, int32_t n_sets, ap_handle *out) {
  if (!out) return AP_ERR_ARG;
  *out = nullptr;
  if (!descs || n_sets < 1 || n_sets > AP_MAX_SETS) return AP_ERR_ARG;
  for (int s = 0; s < n_sets; ++s) {
    int rc = check_desc(descs[s]);
    if (rc != AP_OK) return rc;
  }
  ap_handle_s *h = new (std::nothrow) ap_handle_s();
  if (!h) return AP_ERR_ARG;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) !=
          cudaSuccess) {
    delete h;
    return AP_ERR_CUDA;
  }
  h->n_sets = n_sets;
  h->descs.assign(descs, descs + n_sets);
  h->pd.resize(n_sets);
  h->pf.resize(n_sets);
  h->uniform_kind = descs[0].kind;
  for (int s = 0; s < n_sets; ++s) {
    derive(descs[s], h->pd[s], h->pf[s]);
    if (descs[s].kind != h->uniform_kind) h->uniform_kind = -1;
  }
  const size_t bd = sizeof(Pulse<double>) * n_sets, bf = sizeof(Pulse<float>) * n_sets;
  if (cudaMalloc(&h->d_pd, bd) != cudaSuccess || cudaMalloc(&h->d_pf, bf) != cudaSuccess ||
      cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemcpy(h->d_pd, h->pd.data(), bd, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_pf, h->pf.data(), bf, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaFree(h->d_pd);
    cudaFree(h->d_pf);
    cudaFree(h->d_status);
    delete h;
    return AP_ERR_CUDA;
  }
  *out = h;
  return AP_OK;
}

void ap_destroy(ap_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->d_pd);
  cudaFree(h->d_pf);
  cudaFree(h->d_status);
  delete h;
}

int ap_num_sets(ap_handle h) { return h ? h->n_sets : AP_ERR_ARG; }

int ap_set_launch(ap_handle h, const ap_launch_cfg *cfg) {
  if (!h) return AP_ERR_ARG;
  if (!cfg) {
    h->shape = apt::LaunchShape{0, 0, 0, 0, 0};
    return AP_OK;
  }
  if (cfg->block != 0 && (cfg->block < 32 || cfg->block > 256 || (cfg->block & 31))) return AP_ERR_ARG;
  if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 64) return AP_ERR_ARG;
  if (cfg->grid_cache < 0 || cfg->grid_cache > 2) return AP_ERR_ARG;
  if (cfg->pairs != 0 && cfg->pairs != 1) return AP_ERR_ARG;
  if (cfg->tile < 0 || cfg->tile > (1 << 24)) return AP_ERR_ARG;
  h->shape = apt::LaunchShape{cfg->block, cfg->blocks_per_sm, cfg->grid_cache, cfg->pairs, cfg->tile};
  return AP_OK;
}

int ap_eval_fields(ap_handle h, int32_t set, const double *xyzt, int64_t n, double *EB_out,
                   int32_t precision, void *stream) {
  if (!h || set < 0 || set >= h->n_sets || n < 0) return AP_ERR_ARG;
  if (precision < AP_FP64 || precision > AP_FP32_PHASEFF) return AP_ERR_ARG;
  if (n == 0) return AP_OK;
  if (!xyzt || !EB_out) return AP_ERR_ARG;
  int rc = current_device_matches(h);
  if (rc != AP_OK) return rc;
  apt::EvalArgs a{xyzt, n, EB_out, h->d_status};
  return apt::launch_eval(h->descs[set].kind, precision, h->pd[set], h->pf[set], a, stream);
}

namespace {

// Analytic E1/B1 (current = 0) or J1 (current = 1) on the staggered nodes.
int eval_nodes_common(ap_handle h, int32_t set, const ap_yee_grid *g, double t, int32_t accumulate,
                      int32_t precision, void *stream, int current) {
  if (!h || !g || set < 0 || set >= h->n_sets) return AP_ERR_ARG;
  if (current && (h->descs[set].kind != AP_PLANE || g->f[3] || g->f[4] || g->f[5])) return AP_ERR_ARG;
  if (precision < AP_FP64 || precision > AP_FP32_PHASEFF) return AP_ERR_ARG;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !std::isfinite(t)) return AP_ERR_ARG;
  // node indices (and index + grid stride) are exact in float; the node
  // count fits the index arithmetic
  if (g->nx > (1 << 23) || g->ny > (1 << 23) || g->nz > (1 << 23)) return AP_ERR_ARG;
  if ((double)g->nx * (double)g->ny * (double)g->nz > 1e12) return AP_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(g->lo[a]) || !std::isfinite(g->d[a]) || g->d[a] < 0.0) return AP_ERR_ARG;
  const uintptr_t mask = g->f64 ? 7u : 3u;
  bool any = false;
  for (int c = 0; c < 6; ++c) {
    if (!g->f[c]) continue;
    if ((reinterpret_cast<uintptr_t>(g->f[c]) & mask) != 0) return AP_ERR_ALIGN;
    any = true;
  }
  int rc = current_device_matches(h);
  if (rc != AP_OK) return rc;
  if (!any) return AP_OK;
  apt::NodeArgs a;
  std::memset(&a, 0, sizeof(a));
  // plane waves: E_z = B_z = 0, and E_x, B_y (E_y, B_x) vanish with p_x (p_y);
  // adding an identically zero component is skipped
  const apt::Pulse<double> &P = h->pd[set];
  const bool px0 = P.px_re == 0.0 && P.px_im == 0.0, py0 = P.py_re == 0.0 && P.py_im == 0.0;
  const bool zero[6] = {px0, py0, true, py0, px0, true};
  for (int c = 0; c < 6; ++c) {
    a.f[c] = g->f[c];
    if (!g->f[c]) continue;
    if (accumulate && P.kind == AP_PLANE && zero[c]) continue;
    a.comp[a.n_comp++] = c;
  }
  if (a.n_comp == 0) return AP_OK;
  a.nx = g->nx;
  a.ny = g->ny;
  a.nz = g->nz;
  a.f64 = g->f64 ? 1 : 0;
  a.accumulate = accumulate ? 1 : 0;
  for (int c = 0; c < 3; ++c) {
    a.lo[c] = g->lo[c];
    a.d[c] = g->d[c];
    a.lo_hi[c] = (float)g->lo[c];
    a.lo_lo[c] = (float)(g->lo[c] - (double)a.lo_hi[c]);
    a.d_hi[c] = (float)g->d[c];
    a.d_lo[c] = (float)(g->d[c] - (double)a.d_hi[c]);
  }
  a.t = t;
  a.sm_count = h->sm_count;
  a.current = current;
  return apt::launch_nodes(h->descs[set].kind, precision, h->pd[set], h->pf[set], a, stream);
}

}  // namespace

int ap_eval_nodes(ap_handle h, int32_t set, const ap_yee_grid *g, double t, int32_t accumulate,
                  int32_t precision, void *stream) {
  return eval_nodes_common(h, set, g, t, accumulate, precision, stream, 0);
}

int ap_eval_current(ap_handle h, int32_t set, const ap_yee_grid *g, double t, int32_t accumulate,
                    int32_t precision, void *stream) {
  return eval_nodes_common(h, set, g, t, accumulate, precision, stream, 1);
}

int ap_gather_push(ap_handle h, const ap_particles *p, const ap_grid *g, double t0, double dt,
                   int64_t n_steps, int32_t precision, const ap_diag *diag, void *stream) {
  if (!h) return AP_ERR_ARG;
  int rc = current_device_matches(h);
  if (rc != AP_OK) return rc;
  apt::PushArgs a;
  rc = fill_push_args(h, p, g, t0, dt, n_steps, precision, diag, 1, a, stream);
  if (rc != AP_OK) return rc;
  if (p->n == 0 || n_steps == 0) return AP_OK;
  return apt::launch_push(h->descs[0].kind, precision, h->pd[0], h->pf[0], a, stream);
}

size_t ap_batch_workspace_bytes(ap_handle h) { return h ? 256 : 0; }

int ap_gather_push_batched(ap_handle h, const ap_particles *p, const ap_grid *g, double t0,
                           double dt, int64_t n_steps, int32_t precision, const ap_diag *diag,
                           void *workspace, size_t ws_bytes, void *stream) {
  if (!h || !p) return AP_ERR_ARG;
  int rc = current_device_matches(h);
  if (rc != AP_OK) return rc;
  if (p->n_sets != h->n_sets || !p->set_offsets) return AP_ERR_ARG;
  if (h->uniform_kind < 0) return AP_ERR_UNSUPPORTED;
  if (!workspace || ws_bytes < ap_batch_workspace_bytes(h)) return AP_ERR_WORKSPACE;
  if (!aligned16(workspace) || !aligned16(p->set_offsets)) return AP_ERR_ALIGN;
  apt::BatchArgs ba;
  std::memset(&ba, 0, sizeof(ba));
  rc = fill_push_args(h, p, g, t0, dt, n_steps, precision, diag, h->n_sets, ba.base, stream);
  if (rc != AP_OK) return rc;
  if (n_steps == 0) return AP_OK;
  ba.base.shape.block = h->shape.block > 0 ? h->shape.block : 128;
  // particles per tile: a multiple of what one block carries per pass
  const int per_pass = ba.base.shape.block * (h->shape.pairs ? 2 : 1);
  if (h->shape.tile > 0 && h->shape.tile % per_pass != 0) return AP_ERR_ARG;
  ba.set_offsets = reinterpret_cast<const long long *>(p->set_offsets);
  ba.n_sets = h->n_sets;
  ba.tile_counter = static_cast<unsigned int *>(workspace);
  ba.tile = h->shape.tile > 0 ? h->shape.tile : per_pass;
  if (cudaMemsetAsync(workspace, 0, sizeof(unsigned int), static_cast<cudaStream_t>(stream)) !=
      cudaSuccess)
    return AP_ERR_CUDA;
  return apt::launch_batch(h->uniform_kind, precision, h->d_pd, h->d_pf, ba, stream);
}

int ap_batch_graph_create(ap_handle h, const ap_particles *p, const ap_grid *g, double t0,
                          double dt, int64_t n_steps, int32_t precision, const ap_diag *diag,
                          void *workspace, size_t ws_bytes, void *stream, ap_graph *out) {
  if (!out) return AP_ERR_ARG;
  *out = nullptr;
  if (!stream) return AP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return AP_ERR_CUDA;
  int rc = ap_gather_push_batched(h, p, g, t0, dt, n_steps, precision, diag, workspace, ws_bytes, stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (rc != AP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess || !graph) return AP_ERR_CUDA;
  ap_graph_s *gr = new (std::nothrow) ap_graph_s();
  if (!gr) {
    cudaGraphDestroy(graph);
    return AP_ERR_ARG;
  }
  gr->graph = graph;
  if (cudaGraphInstantiate(&gr->exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    delete gr;
    return AP_ERR_CUDA;
  }
  *out = gr;
  return AP_OK;
}

int ap_graph_launch(ap_graph gr, void *stream) {
  if (!gr || !gr->exec) return AP_ERR_ARG;
  return cudaGraphLaunch(gr->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? AP_OK
                                                                                     : AP_ERR_CUDA;
}

void ap_graph_destroy(ap_graph gr) {
  if (!gr) return;
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  delete gr;
}

int ap_sync_status(ap_handle h, void *stream) {
  if (!h) return AP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  if (cudaMemcpyAsync(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemsetAsync(h->d_status, 0, sizeof(int), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return AP_ERR_CUDA;
  if (v & apt::kStatusNonfinite) return AP_ERR_NONFINITE;
  return AP_OK;
}

}  // extern "C"

namespace {

// Validates a line description and fills the kernel arguments.
int line_args(const ap_line1d *y, int64_t n_steps, int32_t precision, apt::LineArgs *a) {
  if (!y || n_steps < 0 || y->n_lines < 0) return AP_ERR_ARG;
  if (precision != AP_FP64 && precision != AP_FP32_PHASEFF) return AP_ERR_ARG;
  const int max_nodes = precision == AP_FP64 ? AP_LINE1D_MAX_NODES_F64 : AP_LINE1D_MAX_NODES_F32;
  if (y->nz < 2 || y->nz > max_nodes) return AP_ERR_ARG;
  if (!(y->dz > 0.0) || !(y->dt > 0.0) || !(y->dz < 1e300) || !(y->dt < 1e300)) return AP_ERR_ARG;
  if (!(y->omega_p >= 0.0) || !std::isfinite(y->omega_p) || !std::isfinite(y->z0)) return AP_ERR_ARG;
  if (y->n_lines > 0 && (!y->E || !y->B || !y->J)) return AP_ERR_ARG;
  const uintptr_t mask = precision == AP_FP64 ? 7u : 3u;
  const uintptr_t bits = reinterpret_cast<uintptr_t>(y->E) | reinterpret_cast<uintptr_t>(y->B) |
                         reinterpret_cast<uintptr_t>(y->J) | reinterpret_cast<uintptr_t>(y->wp2);
  if ((bits & mask) != 0) return AP_ERR_ALIGN;
  std::memset(a, 0, sizeof(*a));
  a->E = y->E;
  a->B = y->B;
  a->J = y->J;
  a->wp2 = y->wp2;
  a->nz = y->nz;
  a->n_lines = y->n_lines;
  a->dz = y->dz;
  a->dt = y->dt;
  a->omega_p2 = y->omega_p * y->omega_p;
  a->z0 = y->z0;
  a->z0_hi = (float)y->z0;
  a->z0_lo = (float)(y->z0 - (double)a->z0_hi);
  a->dz_hi = (float)y->dz;
  a->dz_lo = (float)(y->dz - (double)a->dz_hi);
  a->n_steps = n_steps;
  return AP_OK;
}

}  // namespace

int ap_plasma1d_run(const ap_line1d *y, int64_t n_steps, int32_t precision, void *stream) {
  apt::LineArgs a;
  const int rc = line_args(y, n_steps, precision, &a);
  if (rc != AP_OK) return rc;
  if (y->n_lines == 0 || n_steps == 0) return AP_OK;
  static const Pulse<double> unused_d{};
  static const Pulse<float> unused_f{};
  return apt::launch_line(false, precision, unused_d, unused_f, a, stream);
}

int ap_apt1d_run(ap_handle h, int32_t set, const ap_line1d *y, double t0, int64_t n_steps,
                 int32_t precision, void *stream) {
  if (!h || set < 0 || set >= h->n_sets || !std::isfinite(t0)) return AP_ERR_ARG;
  const ap_pulse_desc &d = h->descs[set];
  if (d.kind != AP_PLANE || d.pol != AP_LIN_X) return AP_ERR_ARG;
  // float-float time levels: 2 n + 1 exact in float
  if (precision == AP_FP32_PHASEFF && n_steps >= (1 << 23)) return AP_ERR_ARG;
  if (precision == AP_FP32_PHASEFF && y && y->nz > AP_APT1D_MAX_NODES_F32) return AP_ERR_ARG;
  apt::LineArgs a;
  int rc = line_args(y, n_steps, precision, &a);
  if (rc != AP_OK) return rc;
  rc = current_device_matches(h);
  if (rc != AP_OK) return rc;
  if (y->n_lines == 0 || n_steps == 0) return AP_OK;
  a.t0 = t0;
  return apt::launch_line(true, precision, h->pd[set], h->pf[set], a, stream);
}
