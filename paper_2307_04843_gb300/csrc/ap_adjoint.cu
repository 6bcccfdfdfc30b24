// ap_adjoint.cu -- discrete adjoint of the gather + Boris push (row a13).
//
// Objective per set s: J_s = (1/N_s) sum_{i in s} gamma_i(T).  Gradients with
// respect to the pulse parameters theta = (a0, w0, z_f, beta_f) of every set
// (beta_f only for the closed-form flying focus; zero otherwise), by the
// exact reverse of the discrete forward map (the same float-float or double
// arithmetic as ap_gather_push):
//
//   forward:  x^{n+1} = x^n + dt u^{n+1}/gamma^{n+1},  u^{n+1} = Boris(u^n, E(x^n), B(x^n))
//   reverse:  lu'  = lu^{n+1} + dt/gamma' (lx - v' (v'.lx))         (position update)
//             (lu^n, lE, lB) = Boris^T(lu')                          (hand-written VJP)
//             lx^n = lx^{n+1} + (dF/dx)^T (lE, lB),  g += (dF/dtheta)^T (lE, lB)
//
// with seed lu^N = u^N / (gamma^N N_s), lx^N = 0.  dF/dx and dF/dtheta are
// the derivatives in (x, y, z - z_f, w0, beta_f): in closed form for the
// Gaussian beam and the closed-form flying focus (beam_reverse), and from
// the field functions instantiated with forward-mode dual numbers for the
// other kinds; a0 enters linearly (dF/da0 = F / a0) and z_f only through
// z - z_f (dF/dz_f = -dF/dz for the analytic part).
//
// Memory: one persistent launch; every resident thread slot pushes its
// particle forward storing a checkpoint every K steps, then sweeps the
// segments backwards, recomputing each from its checkpoint into a per-slot
// tape.  Checkpoints and tapes live in the caller's workspace, sized by the
// number of resident thread slots, not by the number of particles.
#include <cuda_runtime.h>

#include <cstring>

#include "ap_dual.cuh"
#include "ap_kernels.cuh"

namespace apt {

constexpr int kAdjBlock = 128;
constexpr int kAdjBlocksPerSm = 4;
constexpr int kAdjMaxK = 256;
constexpr int kAdjStateBytes = 48;  // one saved state: 6 doubles or 9 floats
// tangents: x, y, z - z_f, w0 and, for the closed-form flying focus only,
// beta_f (the other kinds do not depend on it: a fifth tangent would be
// dead arithmetic in every dual operation)
template <int KIND>
__host__ __device__ constexpr int tangents() { return KIND == AP_FLYING_CF ? 5 : 4; }
constexpr int kNp = 4;   // parameters: a0, w0, z_f, beta_f

// Pulse view with the w0-dependent constants as duals (tangent slot 3) and,
// for the closed-form flying focus, the beta_f-dependent ones (slot 4).
template <typename R, int NT>
struct PulseAD {
  static constexpr bool kHasPlasma = true;
  int32_t kind, pol, env, lon, lg_p, lg_al, lg_sgn, sg_order, plasma;
  R amp, bratio, lonE, lonB, env_a, env_b, px_re, px_im, py_re, py_im;
  R fdc, inv_w, lg_c1, lg_c2;  // plane wave in a plasma (Sec. 4, Eq. b_corr_t)
  R lg_alf;                    // |l| as a number
  R lg_r[6][kLgMaxP];
  Dual<R, NT> inv_w0sq, inv_zR, lg_pref, beta_f;
};

template <int NT, typename R>
__device__ __forceinline__ PulseAD<R, NT> make_ad(const Pulse<R> &P) {
  using D = Dual<R, NT>;
  PulseAD<R, NT> A;
  A.kind = P.kind; A.pol = P.pol; A.env = P.env; A.lon = P.lon;
  A.lg_p = P.lg_p; A.lg_al = P.lg_al; A.lg_sgn = P.lg_sgn; A.sg_order = P.sg_order;
  A.plasma = P.plasma; A.fdc = P.fdc; A.inv_w = P.inv_w; A.lg_c1 = P.lg_c1; A.lg_c2 = P.lg_c2;
  A.lg_alf = P.lg_alf;
  A.amp = P.amp_unit;  // unit a0: the physical field is a0 times this one
  A.bratio = P.bratio; A.lonE = P.lonE; A.lonB = P.lonB;
  A.env_a = P.env_a; A.env_b = P.env_b;
  A.px_re = P.px_re; A.px_im = P.px_im; A.py_re = P.py_re; A.py_im = P.py_im;
  for (int r = 0; r < 6; ++r)
    for (int k = 0; k < kLgMaxP; ++k) A.lg_r[r][k] = P.lg_r[r][k];
  const R iw = P.inv_w0;
  // d(1/w0^2)/dw0 = -2/w0^3; z_R ~ w0^2; (sqrt2/w0)^|l| ~ w0^-|l|
  A.inv_w0sq = D::seed(P.inv_w0sq, 3, R(-2) * P.inv_w0sq * iw);
  A.inv_zR = D::seed(P.inv_zR, 3, R(-2) * P.inv_zR * iw);
  A.lg_pref = D::seed(P.lg_pref, 3, -R(P.lg_al) * P.lg_pref * iw);
  A.beta_f = D(P.beta_f);
  if constexpr (NT == 5) {
    // closed-form flying focus: zeta = ((z - z_f) - beta_f (t - t_f)) / z_R',
    // 1/z_R' = 1 / ((1 - beta_f) z_R) -> d/dbeta_f = (1/z_R') / (1 - beta_f)
    A.beta_f.d[4] = R(1);
    A.inv_zR.d[4] = P.inv_zR * P.inv_1mb;
  }
  return A;
}

// Saved particle state (checkpoints and tape), strided by thread slot.
template <int PREC>
struct StateIO;

template <>
struct StateIO<AP_FP32_PHASEFF> {
  static constexpr int W = 9;
  __device__ static void put(float *base, size_t stride, const Pos<AP_FP32_PHASEFF> &p,
                             const float u[3]) {
    base[0 * stride] = p.x.hi; base[1 * stride] = p.x.lo;
    base[2 * stride] = p.y.hi; base[3 * stride] = p.y.lo;
    base[4 * stride] = p.z.hi; base[5 * stride] = p.z.lo;
    base[6 * stride] = u[0]; base[7 * stride] = u[1]; base[8 * stride] = u[2];
  }
  __device__ static void get(const float *base, size_t stride, Pos<AP_FP32_PHASEFF> &p, float u[3]) {
    p.x.hi = base[0 * stride]; p.x.lo = base[1 * stride];
    p.y.hi = base[2 * stride]; p.y.lo = base[3 * stride];
    p.z.hi = base[4 * stride]; p.z.lo = base[5 * stride];
    u[0] = base[6 * stride]; u[1] = base[7 * stride]; u[2] = base[8 * stride];
  }
  using T = float;
};

template <>
struct StateIO<AP_FP64> {
  static constexpr int W = 6;
  __device__ static void put(double *base, size_t stride, const Pos<AP_FP64> &p, const double u[3]) {
    base[0 * stride] = p.x; base[1 * stride] = p.y; base[2 * stride] = p.z;
    base[3 * stride] = u[0]; base[4 * stride] = u[1]; base[5 * stride] = u[2];
  }
  __device__ static void get(const double *base, size_t stride, Pos<AP_FP64> &p, double u[3]) {
    p.x = base[0 * stride]; p.y = base[1 * stride]; p.z = base[2 * stride];
    u[0] = base[3 * stride]; u[1] = base[4 * stride]; u[2] = base[5 * stride];
  }
  using T = double;
};

struct AdjArgs {
  PushArgs base;              // particles (read only), grid, t0, dt, n_steps, status
  const long long *set_offsets;  // nullptr: one set [0, n)
  int n_sets;
  int K;                      // steps per segment
  int n_seg;
  unsigned int *tile_counter;
  void *ckpt;                 // [n_seg][W][nslots]
  void *tape;                 // [K][W][nslots]
  long long nslots;
  double *dJ;                 // [n_sets][AP_NPARAM]
  double *J;                  // [n_sets] or null
};

template <typename R>
struct GridGrad {
  R v[6];
  R g[6][3];
};

// Trilinear value and gradient from the cached cell (zero gradient along an
// axis on which the position is clamped to the box).
template <typename R>
__device__ __forceinline__ void grid_value_grad(const GridView &g, GridCache<R> &gc, R x, R y, R z,
                                                GridGrad<R> &out) {
  R E[3] = {R(0), R(0), R(0)}, B[3] = {R(0), R(0), R(0)};
  grid_gather<R>(g, gc, x, y, z, E, B);  // refreshes the cache and the weights
  R idd[3], off[3];
  if constexpr (std::is_same<R, double>::value) {
    for (int a = 0; a < 3; ++a) { idd[a] = g.inv_d_d[a]; off[a] = g.off_d[a]; }
  } else {
    for (int a = 0; a < 3; ++a) { idd[a] = g.inv_d[a]; off[a] = g.off[a]; }
  }
  // unclamped grid coordinates: the gradient vanishes along clamped axes
  const R fxr = fma(x, idd[0], off[0]), fyr = fma(y, idd[1], off[1]), fzr = fma(z, idd[2], off[2]);
  const R wx = gc.wx, wy = gc.wy, wz = gc.wz;
  const R ux = R(1) - wx, uy = R(1) - wy, uz = R(1) - wz;
  const R sx = (fxr >= R(0) && fxr <= R(g.nx - 1)) ? idd[0] : R(0);
  const R sy = (fyr >= R(0) && fyr <= R(g.ny - 1)) ? idd[1] : R(0);
  const R sz = (fzr >= R(0) && fzr <= R(g.nz - 1)) ? idd[2] : R(0);
  out.v[0] = E[0]; out.v[1] = E[1]; out.v[2] = E[2];
  out.v[3] = B[0]; out.v[4] = B[1]; out.v[5] = B[2];
  for (int c = 0; c < 6; ++c) {
    // raw corners k[cx + 2 cy + 4 cz]; derivative of the trilinear weights
    const R *k = gc.c[c];
    R dfx = (k[1] - k[0]) * uy * uz + (k[3] - k[2]) * wy * uz + (k[5] - k[4]) * uy * wz +
            (k[7] - k[6]) * wy * wz;
    R dfy = (k[2] - k[0]) * ux * uz + (k[3] - k[1]) * wx * uz + (k[6] - k[4]) * ux * wz +
            (k[7] - k[5]) * wx * wz;
    R dfz = (k[4] - k[0]) * ux * uy + (k[5] - k[1]) * wx * uy + (k[6] - k[2]) * ux * wy +
            (k[7] - k[3]) * wx * wy;
    out.g[c][0] = dfx * sx;
    out.g[c][1] = dfy * sy;
    out.g[c][2] = dfz * sz;
  }
}

template <int KIND, typename R, int NT>
__device__ __forceinline__ void fields_ad(const PulseAD<R, NT> &A, const Local<Dual<R, NT>> &L,
                                          Dual<R, NT> E[3], Dual<R, NT> B[3]) {
  if constexpr (KIND == AP_PLANE) fields_plane(A, L, E, B);
  else if constexpr (KIND == AP_GAUSS) fields_gauss(A, L, E, B);
  else if constexpr (KIND == AP_FLYING_CF) fields_gauss<true>(A, L, E, B);
  else fields_lg(A, L, E, B);
}

// Logarithmic derivative Gamma'/Gamma of the envelope at eta, given the
// factor `mul` that `envelope` returned (zero outside the sin^2 window and
// for a continuous wave).  SIN2: Gamma = cos^2(env_a eta), so -2 env_a
// tan(env_a eta); GAUSS: Gamma = 2^(-env_a eta^2); SGAUSS: Gamma =
// 2^(-env_b u^(2g)), u = env_a eta.
template <typename R>
__device__ __forceinline__ R unless_zero(R v, R m) { return m == R(0) ? R(0) : v; }
__device__ __forceinline__ F2 unless_zero(F2 v, F2 m) {
  return F2(m.x == 0.0f ? 0.0f : v.x, m.y == 0.0f ? 0.0f : v.y);
}

template <class PT, typename R>
__device__ __forceinline__ R envelope_dlog(const PT &P, R eta, R mul) {
  constexpr double kLn2 = 0.69314718055994531;
  switch (P.env) {
    case AP_ENV_SIN2: {
      // evaluated in both halves of a pair, each cleared where its factor is 0
      R s, c;
      sincos_r(eta * P.env_a, &s, &c);
      return unless_zero(R(-2) * P.env_a * s * rcp_r(c), mul);
    }
    case AP_ENV_GAUSS:
      return R(-2 * kLn2) * P.env_a * eta;
    case AP_ENV_SGAUSS: {
      const R u = eta * P.env_a;
      const R s = u * u;
      R p = R(1);  // s^(g-1)
      for (int i = 1; i < P.sg_order; ++i) p *= s;
      return R(-2 * kLn2) * P.env_b * R(P.sg_order) * P.env_a * u * p;
    }
    default:
      return R(0);
  }
}

// The reverse of one Boris step and position update, given the fields F at
// the step's position: from the adjoints lx, lu of the state after the step,
// the cotangent Fb of the fields (E, B), with lu updated to the momentum
// adjoint before the step (lx changes only through the fields:
// lx += (dF/dx)^T Fb).  Generic over the arithmetic type (float, double, or
// the packed pair of the two-particle kernel); adv_xy = 0 holds the
// transverse position (1D-3V).
template <typename R>
__device__ __forceinline__ void boris_cotangent(const R F[6], const R u[3], R dt, R adv_xy,
                                                const R lx[3], R lu[3], R Fb[6]) {
  const R h = R(-0.5) * dt;
  const R E[3] = {F[0], F[1], F[2]}, B[3] = {F[3], F[4], F[5]};
  // Boris forward intermediates
  R am[3] = {fma(h, E[0], u[0]), fma(h, E[1], u[1]), fma(h, E[2], u[2])};
  R ig = rsqrt_r(R(1) + am[0] * am[0] + am[1] * am[1] + am[2] * am[2]);
  R tau[3] = {h * ig * B[0], h * ig * B[1], h * ig * B[2]};
  R tt = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
  R f = R(2) * rcp_r(R(1) + tt);
  R s[3] = {f * tau[0], f * tau[1], f * tau[2]};
  R p[3] = {am[0] + (am[1] * tau[2] - am[2] * tau[1]), am[1] + (am[2] * tau[0] - am[0] * tau[2]),
            am[2] + (am[0] * tau[1] - am[1] * tau[0])};
  R bq[3] = {am[0] + (p[1] * s[2] - p[2] * s[1]), am[1] + (p[2] * s[0] - p[0] * s[2]),
             am[2] + (p[0] * s[1] - p[1] * s[0])};
  R un[3] = {fma(h, E[0], bq[0]), fma(h, E[1], bq[1]), fma(h, E[2], bq[2])};
  R ign = rsqrt_r(R(1) + un[0] * un[0] + un[1] * un[1] + un[2] * un[2]);
  R v[3] = {un[0] * ign, un[1] * ign, un[2] * ign};
  // position update: x'_k = x_k + dt_k u'_k / gamma', dt_k = (dt_xy, dt_xy, dt)
  // (dt_xy = 0 for a 1D-3V set): d x'_k / d u'_j = dt_k ign (delta_kj - v_k v_j)
  const R dtk[3] = {dt * adv_xy, dt * adv_xy, dt};
  R vl = dtk[0] * v[0] * lx[0] + dtk[1] * v[1] * lx[1] + dtk[2] * v[2] * lx[2];
  R ub[3];
  for (int k = 0; k < 3; ++k) ub[k] = lu[k] + ign * (dtk[k] * lx[k] - v[k] * vl);
  // Boris reverse
  R Eb[3], Bb[3], ab[3], pb[3], sbar[3], tb[3];
  for (int k = 0; k < 3; ++k) Eb[k] = h * ub[k];
  // b = a + p x s
  pb[0] = s[1] * ub[2] - s[2] * ub[1];
  pb[1] = s[2] * ub[0] - s[0] * ub[2];
  pb[2] = s[0] * ub[1] - s[1] * ub[0];
  sbar[0] = ub[1] * p[2] - ub[2] * p[1];
  sbar[1] = ub[2] * p[0] - ub[0] * p[2];
  sbar[2] = ub[0] * p[1] - ub[1] * p[0];
  // p = a + a x tau
  ab[0] = ub[0] + pb[0] + (tau[1] * pb[2] - tau[2] * pb[1]);
  ab[1] = ub[1] + pb[1] + (tau[2] * pb[0] - tau[0] * pb[2]);
  ab[2] = ub[2] + pb[2] + (tau[0] * pb[1] - tau[1] * pb[0]);
  tb[0] = pb[1] * am[2] - pb[2] * am[1];
  tb[1] = pb[2] * am[0] - pb[0] * am[2];
  tb[2] = pb[0] * am[1] - pb[1] * am[0];
  // s = f tau, f = 2 / (1 + tau^2)
  R ts = tau[0] * sbar[0] + tau[1] * sbar[1] + tau[2] * sbar[2];
  for (int k = 0; k < 3; ++k) tb[k] += f * sbar[k] - f * f * tau[k] * ts;
  // tau = h ig B
  R igb = h * (B[0] * tb[0] + B[1] * tb[1] + B[2] * tb[2]);
  for (int k = 0; k < 3; ++k) Bb[k] = h * ig * tb[k];
  // ig = (1 + a^2)^(-1/2)
  R c3 = -ig * ig * ig * igb;
  for (int k = 0; k < 3; ++k) ab[k] += c3 * am[k];
  for (int k = 0; k < 3; ++k) {
    Eb[k] += h * ab[k];
    lu[k] = ab[k];
  }
  for (int k = 0; k < 3; ++k) {
    Fb[k] = Eb[k];
    Fb[k + 3] = Bb[k];
  }
}

// The grid's share of a reverse step: its interpolated fields join the
// analytic ones before the Boris reverse, and its gradient joins the
// position adjoint after it.
struct NoGridPart {
  template <typename R>
  __device__ __forceinline__ void add(R *) const {}
  template <typename R>
  __device__ __forceinline__ void contract(const R *, R *) const {}
};
template <typename R>
struct GridPart {
  GridGrad<R> gg;
  __device__ __forceinline__ void add(R F[6]) const {
    for (int c = 0; c < 6; ++c) F[c] += gg.v[c];
  }
  __device__ __forceinline__ void contract(const R Fb[6], R lx[3]) const {
    for (int c = 0; c < 6; ++c)
      for (int k = 0; k < 3; ++k) lx[k] += Fb[c] * gg.g[c][k];
  }
};

// One reverse step of the Gaussian beam (MOVING: the closed-form flying
// focus), with the field derivatives in the directions j = (x, y, z - z_f,
// w0[, beta_f]) in closed form rather than by dual numbers, each contracted
// with the field cotangent Fb as soon as it is formed (no Jacobian is kept).
// The value part is the arithmetic of gauss_z and gauss_xy.  With G the
// amplitude times the envelope and a = r^2/w0^2, the profile is
// U0 = G e^{i psi} exp(-a q), U = q U0 and W = q U (the longitudinal terms'
// factor), and dq/dzeta = i q^2; so every derivative is a complex factor
// times U or W:
//   dU/dj = U alpha_j,  alpha_j = i q (1 - a q) zeta_j - a_j q + L1 eta_j + i psi_j,
//   dW/dj = W beta_j,   beta_j = alpha_j + i q zeta_j,
// L1 = Gamma'/Gamma, where zeta_j, a_j, eta_j, psi_j are the derivatives of
// zeta, a, eta = T - (z - z_f)/v_g and psi = C - k (z - z_f).  The fields
// are linear in U and W (finish_beam), with the longitudinal terms also
// linear in x, y and g = -2/w0^2, whose derivatives add those terms at unit
// x, at unit y, and times g'/g = -2/w0.  Order: the value and the factors
// the derivatives share, the Boris reverse for Fb, then Fb . dF/dj per
// direction.  F = a0 f with f the unit-a0 fields: dF/da0 = f, d/dz_f =
// -d/d(z - z_f).
template <int POL, bool LON, bool MOVING, class PT, typename R, class GP>
__device__ __forceinline__ void beam_reverse_t(const PT &P, const Local<R> &L, R a0, const R u[3],
                                               R dt, R adv_xy, R lx[3], R lu[3], R gr[kNp],
                                               const GP &grid) {
  constexpr int NT = MOVING ? 5 : 4;
  R mul, l2;
  envelope(P, L.eta, mul, l2);
  R zeta;
  if constexpr (MOVING) zeta = fma(-P.beta_f, L.T, L.dz) * P.inv_zR;
  else zeta = L.dz * P.inv_zR;
  const R inv = rcp_r(fma(zeta, zeta, R(1)));
  const Cx<R> q{inv, zeta * inv};
  const R x = L.x, y = L.y;
  const R a = (x * x + y * y) * P.inv_w0sq;
  const R mag = (P.amp_unit * mul) * exp2_r(fma(a * q.re, R(-kLog2e), l2));
  const R ang = reduce_angle<R>(L.psi - a * q.im);
  R sn, cs;
  sincos_r(ang, &sn, &cs);
  const Cx<R> U = cmul(q, Cx<R>{mag * cs, mag * sn});
  const Cx<R> W = cmul(q, U);
  const R g = R(-2) * P.inv_w0sq;
  R f[6], F[6], Fb[6];
  {
    R E[3], B[3];
    finish_beam_pol<POL>(P, x, y, U, W, g, LON, E, B);
    for (int c = 0; c < 3; ++c) {
      f[c] = E[c];
      f[c + 3] = B[c];
    }
  }
  for (int c = 0; c < 6; ++c) F[c] = a0 * f[c];
  grid.add(F);
  boris_cotangent<R>(F, u, dt, adv_xy, lx, lu, Fb);
  grid.contract(Fb, lx);
  R sa0 = Fb[0] * f[0];
  for (int c = 1; c < 6; ++c) sa0 = fma(Fb[c], f[c], sa0);
  // shared factors: i q and i q (1 - a q)
  const Cx<R> iq{-q.im, q.re};
  const Cx<R> Q1 = cmul(iq, Cx<R>{R(1) - a * q.re, -a * q.im});
  const R L1 = envelope_dlog(P, L.eta, mul);
  const R w2 = R(2) * P.inv_w0sq, m2w = R(-2) * P.inv_w0;
  R zj[NT], aj[NT], ej[NT], pj[NT], sj[NT];
  zj[0] = R(0); aj[0] = w2 * x; ej[0] = R(0); pj[0] = R(0);
  zj[1] = R(0); aj[1] = w2 * y; ej[1] = R(0); pj[1] = R(0);
  zj[2] = P.inv_zR; aj[2] = R(0); ej[2] = -P.inv_vg * L1; pj[2] = -R(P.k);
  zj[3] = m2w * zeta; aj[3] = m2w * a; ej[3] = R(0); pj[3] = R(0);
  if constexpr (NT == 5) {
    zj[4] = fma(-L.T, P.inv_zR, zeta * P.inv_1mb);
    aj[4] = R(0); ej[4] = R(0); pj[4] = R(0);
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const Cx<R> al{zj[j] * Q1.re - aj[j] * q.re + ej[j], zj[j] * Q1.im - aj[j] * q.im + pj[j]};
    const Cx<R> be{al.re + zj[j] * iq.re, al.im + zj[j] * iq.im};
    R Ej[3], Bj[3];
    finish_beam_pol<POL>(P, x, y, cmul(U, al), cmul(W, be), g, LON, Ej, Bj);
    R t = Fb[0] * Ej[0];
    t = fma(Fb[1], Ej[1], t);
    t = fma(Fb[2], Ej[2], t);
    t = fma(Fb[3], Bj[0], t);
    t = fma(Fb[4], Bj[1], t);
    sj[j] = fma(Fb[5], Bj[2], t);
  }
  if constexpr (LON) {
    // the longitudinal terms' own x, y and g factors (components E_z, B_z)
    const Cx<R> zero{R(0), R(0)};
    R Ex[3], Bx[3], Ey[3], By[3], Eg[3], Bg[3];
    finish_beam_pol<POL>(P, R(1), R(0), zero, W, g, true, Ex, Bx);
    finish_beam_pol<POL>(P, R(0), R(1), zero, W, g, true, Ey, By);
    finish_beam_pol<POL>(P, x, y, zero, W, g, true, Eg, Bg);
    sj[0] = fma(Fb[2], Ex[2], fma(Fb[5], Bx[2], sj[0]));
    sj[1] = fma(Fb[2], Ey[2], fma(Fb[5], By[2], sj[1]));
    sj[3] = fma(m2w, fma(Fb[2], Eg[2], Fb[5] * Bg[2]), sj[3]);
  }
  lx[0] = fma(a0, sj[0], lx[0]);
  lx[1] = fma(a0, sj[1], lx[1]);
  lx[2] = fma(a0, sj[2], lx[2]);
  gr[0] += sa0;
  gr[1] = fma(a0, sj[3], gr[1]);
  gr[2] = fma(-a0, sj[2], gr[2]);
  if constexpr (NT == 5) gr[3] = fma(a0, sj[4], gr[3]);
}

// beam_reverse_t with the polarisation and the longitudinal switch (uniform
// over a set) selected once rather than in each of its field assemblies.
template <bool MOVING, class PT, typename R, class GP>
__device__ __forceinline__ void beam_reverse(const PT &P, const Local<R> &L, R a0, const R u[3], R dt,
                                             R adv_xy, R lx[3], R lu[3], R gr[kNp], const GP &grid) {
  const bool lon = P.lon != 0;
#define APT_BEAM_REV(POLV)                                                                    \
  if (lon) beam_reverse_t<POLV, true, MOVING>(P, L, a0, u, dt, adv_xy, lx, lu, gr, grid);   \
  else beam_reverse_t<POLV, false, MOVING>(P, L, a0, u, dt, adv_xy, lx, lu, gr, grid)
  switch (P.pol) {
    case AP_LIN_X: APT_BEAM_REV(AP_LIN_X); break;
    case AP_LIN_Y: APT_BEAM_REV(AP_LIN_Y); break;
    case AP_CIRC_P: APT_BEAM_REV(AP_CIRC_P); break;
    default: APT_BEAM_REV(AP_CIRC_M); break;
  }
#undef APT_BEAM_REV
}

// One reverse step.  State before the step (pos, u), step value st, adjoints
// lx, lu of the state after the step (updated in place to the state before),
// gradient accumulators g[0..3] = d/d(a0, w0, z_f, beta_f).
template <int KIND, int PREC, bool GRID>
__device__ __forceinline__ void reverse_step(const Pulse<Real<PREC>> &P,
                                             const PulseAD<Real<PREC>, tangents<KIND>()> &A,
                                             const AdjArgs &aa, const typename TimeBase<PREC>::Step &st,
                                             const Pos<PREC> &pos, const Real<PREC> u[3],
                                             Real<PREC> lx[3], Real<PREC> lu[3], Real<PREC> g[kNp],
                                             GridCache<Real<PREC>> &gc) {
  using R = Real<PREC>;
  constexpr int NT = tangents<KIND>();
  using DR = Dual<R, NT>;
  const R dt = (R)aa.base.dt;
  const R a0 = P.a0;
  const R adv = P.adv_xy;
  // fields with derivatives in (x, y, z - z_f, w0, beta_f)
  const Local<R> L = local_coords<PREC>(P, st, pos);
  auto run = [&](const auto &grid) {
    if constexpr (KIND == AP_GAUSS || KIND == AP_FLYING_CF) {
      beam_reverse<KIND == AP_FLYING_CF>(P, L, a0, u, dt, adv, lx, lu, g, grid);
    } else {
      // the other kinds: dual numbers through the generic field functions
      R F[6], dFx[6][3], dFth[6][kNp];  // field, d/dx, d/d(a0, w0, z_f, beta_f)
      Local<DR> LD;
      LD.x = DR::seed(L.x, 0);
      LD.y = DR::seed(L.y, 1);
      LD.dz = DR::seed(L.dz, 2);
      LD.psi = DR(L.psi);
      LD.psi.d[2] = -R(P.k);  // psi = C - k (z - z_f)
      LD.eta = DR(L.eta);
      LD.eta.d[2] = -P.inv_vg;  // eta = T - (z - z_f) / v_g
      LD.T = DR(L.T);
      LD.phi_hi = DR(R(0));
      LD.phi_lo = DR(R(0));
      DR Ed[3], Bd[3];
      fields_ad<KIND, R, NT>(A, LD, Ed, Bd);
      const DR *Fd[6] = {&Ed[0], &Ed[1], &Ed[2], &Bd[0], &Bd[1], &Bd[2]};
      for (int c = 0; c < 6; ++c) {
        const DR &f = *Fd[c];
        F[c] = a0 * f.v;
        dFx[c][0] = a0 * f.d[0];
        dFx[c][1] = a0 * f.d[1];
        dFx[c][2] = a0 * f.d[2];
        dFth[c][0] = f.v;
        dFth[c][1] = a0 * f.d[3];
        dFth[c][2] = -a0 * f.d[2];
        if constexpr (NT == 5) dFth[c][3] = a0 * f.d[4];
        else dFth[c][3] = R(0);
      }
      grid.add(F);
      R Fb[6];
      boris_cotangent<R>(F, u, dt, adv, lx, lu, Fb);
      grid.contract(Fb, lx);
      for (int c = 0; c < 6; ++c) {
        for (int k = 0; k < 3; ++k) lx[k] += Fb[c] * dFx[c][k];
        for (int k = 0; k < kNp; ++k) g[k] += Fb[c] * dFth[c][k];
      }
    }
  };
  if constexpr (GRID) {
    GridPart<R> gp;
    grid_value_grad<R>(aa.base.grid, gc, L.x, L.y, pos.zr(), gp.gg);
    run(gp);
  } else {
    run(NoGridPart{});
  }
}

template <int KIND, int PREC, bool GRID>
// residency target: kAdjBlocksPerSm blocks for the float kernels without a
// grid, two for the larger FP64 and grid ones (without a minimum the FP64
// kernel was held at 128 registers and spilled)
__global__ void __launch_bounds__(kAdjBlock, (PREC == AP_FP64 || GRID) ? 2 : kAdjBlocksPerSm)
    adjoint_kernel(const Pulse<Real<PREC>> *__restrict__ sets,
                                                            const __grid_constant__ AdjArgs aa) {
  using R = Real<PREC>;
  using IO = StateIO<PREC>;
  using T = typename IO::T;
  __shared__ long long s_tile;
  __shared__ int s_set;
  __shared__ double s_red[32];
  __shared__ StepFF s_steps[kAdjMaxK];
  __shared__ __align__(16) unsigned char s_pulse_raw[sizeof(Pulse<R>)];
  __shared__ long long s_prefix[AP_MAX_SETS + 1];
  // dynamic: the tape state of the next reverse step, copied in while the
  // current one is computed (double buffer [2][W][kAdjBlock], this thread's
  // column only)
  extern __shared__ __align__(16) unsigned char s_adj_dyn[];
  T *s_next = reinterpret_cast<T *>(s_adj_dyn);
  Pulse<R> &P = *reinterpret_cast<Pulse<R> *>(s_pulse_raw);
  const PushArgs &a = aa.base;
  const int Tt = blockDim.x;
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int s = 0; s < aa.n_sets; ++s) {
      s_prefix[s] = acc;
      long long ns = aa.set_offsets ? aa.set_offsets[s + 1] - aa.set_offsets[s] : a.n;
      if (ns < 0) ns = 0;
      acc += (ns + Tt - 1) / Tt;
    }
    s_prefix[aa.n_sets] = acc;
    s_set = -1;
  }
  __syncthreads();
  const long long total = s_prefix[aa.n_sets];
  const size_t slot = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)aa.nslots;
  T *ck = static_cast<T *>(aa.ckpt) + slot;
  T *tp = static_cast<T *>(aa.tape) + slot;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(aa.tile_counter, 1u);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= total) break;
    int lo = 0, hi = aa.n_sets;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (s_prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    const int set = lo;
    if (set != s_set) {
      const int words = (int)(sizeof(Pulse<R>) / 4);
      const uint32_t *src = reinterpret_cast<const uint32_t *>(sets + set);
      uint32_t *dst = reinterpret_cast<uint32_t *>(s_pulse_raw);
      for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0) s_set = set;
    }
    __syncthreads();
    const long long off0 = aa.set_offsets ? aa.set_offsets[set] : 0;
    const long long off1 = aa.set_offsets ? aa.set_offsets[set + 1] : a.n;
    const long long i = off0 + (tile - s_prefix[set]) * Tt + threadIdx.x;
    const bool valid = i >= 0 && i < off1 && i < a.n;
    const double Ns = (double)(off1 - off0);
    // ---- forward pass with checkpoints
    Pos<PREC> pos;
    R u[3] = {R(0), R(0), R(0)};
    pos.load(valid ? a.x[i] : 0.0, valid ? a.y[i] : 0.0, valid ? a.z[i] : 0.0);
    if (valid) {
      u[0] = static_cast<const R *>(a.ux)[i];
      u[1] = static_cast<const R *>(a.uy)[i];
      u[2] = static_cast<const R *>(a.uz)[i];
    }
    TimeBase<PREC> tb;
    tb.init(P, a.t0, a.dt);
    const R dtR = (R)a.dt;
    const R dtxy = dtR * P.adv_xy;
    GridCache<R> gc;
    grid_cache_reset(gc);
    for (int seg = 0; seg < aa.n_seg; ++seg) {
      const long long s0 = (long long)seg * aa.K;
      const int cnt = (int)(a.n_steps - s0 < aa.K ? a.n_steps - s0 : aa.K);
      IO::put(ck + (size_t)seg * IO::W * stride, stride, pos, u);
      if constexpr (PREC == AP_FP32_PHASEFF) {
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) s_steps[k] = tb.at(s0 + k);
        __syncthreads();
      }
      for (int k = 0; k < cnt; ++k) {
        typename TimeBase<PREC>::Step st;
        if constexpr (PREC == AP_FP32_PHASEFF) st = s_steps[k];
        else st = tb.at(s0 + k);
        Local<R> L = local_coords<PREC>(P, st, pos);
        R E[3], B[3];
        analytic_fields<KIND, PREC>(P, L, E, B);
        if constexpr (GRID) grid_gather<R>(a.grid, gc, L.x, L.y, pos.zr(), E, B);
        R ig = boris(u, E, B, dtR);
        pos.advance(u[0] * ig, u[1] * ig, u[2] * ig, dtxy, dtR);
      }
    }
    // ---- objective and seed
    const double gN = sqrt(1.0 + (double)u[0] * u[0] + (double)u[1] * u[1] + (double)u[2] * u[2]);
    R lx[3] = {R(0), R(0), R(0)}, lu[3];
    for (int k = 0; k < 3; ++k) lu[k] = valid ? (R)((double)u[k] / (gN * Ns)) : R(0);
    double Jv = valid ? gN / Ns : 0.0;
    double gacc[kNp] = {0.0, 0.0, 0.0, 0.0};
    const PulseAD<R, tangents<KIND>()> A = make_ad<tangents<KIND>()>(P);
    // ---- reverse sweep over segments
    for (int seg = aa.n_seg - 1; seg >= 0; --seg) {
      const long long s0 = (long long)seg * aa.K;
      const int cnt = (int)(a.n_steps - s0 < aa.K ? a.n_steps - s0 : aa.K);
      IO::get(ck + (size_t)seg * IO::W * stride, stride, pos, u);
      if constexpr (PREC == AP_FP32_PHASEFF) {
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) s_steps[k] = tb.at(s0 + k);
        __syncthreads();
      }
      for (int k = 0; k < cnt; ++k) {
        IO::put(tp + (size_t)k * IO::W * stride, stride, pos, u);
        typename TimeBase<PREC>::Step st;
        if constexpr (PREC == AP_FP32_PHASEFF) st = s_steps[k];
        else st = tb.at(s0 + k);
        Local<R> L = local_coords<PREC>(P, st, pos);
        R E[3], B[3];
        analytic_fields<KIND, PREC>(P, L, E, B);
        if constexpr (GRID) grid_gather<R>(a.grid, gc, L.x, L.y, pos.zr(), E, B);
        R ig = boris(u, E, B, dtR);
        pos.advance(u[0] * ig, u[1] * ig, u[2] * ig, dtxy, dtR);
      }
      // the tape entries this thread just stored are read back by its own
      // asynchronous copies
      __threadfence_block();
      auto stage = [&](int k) {
        const T *src = tp + (size_t)k * IO::W * stride;
#pragma unroll
        for (int w = 0; w < IO::W; ++w) {
          const unsigned dst = (unsigned)__cvta_generic_to_shared(
              s_next + ((k & 1) * IO::W + w) * kAdjBlock + threadIdx.x);
          if constexpr (sizeof(T) == 8) cp_async8(dst, src + (size_t)w * stride);
          else cp_async4(dst, src + (size_t)w * stride);
        }
      };
      R gs[kNp] = {R(0), R(0), R(0), R(0)};
      stage(cnt - 1);
      for (int k = cnt - 1; k >= 0; --k) {
        cp_async_wait_all();
        IO::get(s_next + (k & 1) * IO::W * kAdjBlock + threadIdx.x, kAdjBlock, pos, u);
        if (k > 0) stage(k - 1);
        typename TimeBase<PREC>::Step st;
        if constexpr (PREC == AP_FP32_PHASEFF) st = s_steps[k];
        else st = tb.at(s0 + k);
        reverse_step<KIND, PREC, GRID>(P, A, aa, st, pos, u, lx, lu, gs, gc);
      }
      for (int k = 0; k < kNp; ++k) gacc[k] += (double)gs[k];
    }
    if (!valid) {
      gacc[0] = gacc[1] = gacc[2] = gacc[3] = 0.0;
      Jv = 0.0;
    } else if (!(isfinite(gacc[0]) && isfinite(gacc[1]) && isfinite(gacc[2]) && isfinite(gacc[3]))) {
      atomicOr(a.status, kStatusNonfinite);
    }
    // per-set reduction (every particle of the tile belongs to `set`)
    for (int k = 0; k < kNp; ++k) {
      double t = block_sum(gacc[k], s_red);
      if (threadIdx.x == 0) atomicAdd(aa.dJ + (size_t)set * AP_NPARAM + k, t);
    }
    if (aa.J) {
      double t = block_sum(Jv, s_red);
      if (threadIdx.x == 0) atomicAdd(aa.J + set, t);
    }
    __syncthreads();
  }
}

// ------------------------------------------------- two particles per thread
// The float-float adjoint of the Gaussian kinds without a grid, with each
// thread carrying two particles in the two halves of packed (f32x2) values,
// as the two-particle push does: the forward sweep, the recomputation, the
// closed-form field derivatives and the Boris reverse all run on pairs.  Tiles
// hold 2 kAdjBlock particles of one set (thread t: t and t + kAdjBlock).
// Checkpoints and the tape keep the layout of the one-particle kernel with
// the two particles of a thread side by side: [..][W][thread slots] float2,
// the same bytes for half as many thread slots.
constexpr int kAdjPairBlocksPerSm = 3;  // 156-162 registers, no spills

struct PairIO {
  static constexpr int W = 9;
  __device__ static void put(float2 *b, size_t s, const Pos2 &p, const F2 u[3]) {
    b[0 * s] = make_float2(p.x.hi.x, p.x.hi.y); b[1 * s] = make_float2(p.x.lo.x, p.x.lo.y);
    b[2 * s] = make_float2(p.y.hi.x, p.y.hi.y); b[3 * s] = make_float2(p.y.lo.x, p.y.lo.y);
    b[4 * s] = make_float2(p.dz.hi.x, p.dz.hi.y); b[5 * s] = make_float2(p.dz.lo.x, p.dz.lo.y);
    b[6 * s] = make_float2(u[0].x, u[0].y); b[7 * s] = make_float2(u[1].x, u[1].y);
    b[8 * s] = make_float2(u[2].x, u[2].y);
  }
  __device__ static void get(const float2 *b, size_t s, Pos2 &p, F2 u[3]) {
    float2 v;
    v = b[0 * s]; p.x.hi = F2(v.x, v.y); v = b[1 * s]; p.x.lo = F2(v.x, v.y);
    v = b[2 * s]; p.y.hi = F2(v.x, v.y); v = b[3 * s]; p.y.lo = F2(v.x, v.y);
    v = b[4 * s]; p.dz.hi = F2(v.x, v.y); v = b[5 * s]; p.dz.lo = F2(v.x, v.y);
    v = b[6 * s]; u[0] = F2(v.x, v.y); v = b[7 * s]; u[1] = F2(v.x, v.y);
    v = b[8 * s]; u[2] = F2(v.x, v.y);
  }
};

// reverse_step for a thread's two particles (Gaussian kinds, no grid)
template <int KIND>
__device__ __forceinline__ void reverse_step_pair(const Pulse<float> &P, float dt, const StepFF &st,
                                                  const Pos2 &pos, const F2 u[3], F2 lx[3], F2 lu[3],
                                                  F2 g[kNp]) {
  const Local<F2> L = local_coords2(P, st, pos);
  beam_reverse<KIND == AP_FLYING_CF>(P, L, F2(P.a0), u, F2(dt), F2(P.adv_xy), lx, lu, g, NoGridPart{});
}

template <int KIND>
__global__ void __launch_bounds__(kAdjBlock, kAdjPairBlocksPerSm)
    adjoint_kernel_pair(const Pulse<float> *__restrict__ sets, const __grid_constant__ AdjArgs aa) {
  static_assert(KIND == AP_GAUSS || KIND == AP_FLYING_CF, "kinds with closed-form field derivatives");
  __shared__ long long s_tile;
  __shared__ int s_set;
  __shared__ double s_red[32];
  __shared__ StepFF s_steps[kAdjMaxK];
  __shared__ __align__(16) unsigned char s_pulse_raw[sizeof(Pulse<float>)];
  __shared__ long long s_prefix[AP_MAX_SETS + 1];
  // dynamic: the next reverse step's tape entry, [2][W][kAdjBlock] float2
  extern __shared__ __align__(16) unsigned char s_adj_dyn[];
  float2 *s_next = reinterpret_cast<float2 *>(s_adj_dyn);
  Pulse<float> &P = *reinterpret_cast<Pulse<float> *>(s_pulse_raw);
  const PushArgs &a = aa.base;
  constexpr int kPer = 2 * kAdjBlock;  // particles per tile
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int s = 0; s < aa.n_sets; ++s) {
      s_prefix[s] = acc;
      long long ns = aa.set_offsets ? aa.set_offsets[s + 1] - aa.set_offsets[s] : a.n;
      if (ns < 0) ns = 0;
      acc += (ns + kPer - 1) / kPer;
    }
    s_prefix[aa.n_sets] = acc;
    s_set = -1;
  }
  __syncthreads();
  const long long total = s_prefix[aa.n_sets];
  const size_t slot = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)(aa.nslots / 2);  // thread slots
  float2 *ck = static_cast<float2 *>(aa.ckpt) + slot;
  float2 *tp = static_cast<float2 *>(aa.tape) + slot;
  const float *uxs = static_cast<const float *>(a.ux);
  const float *uys = static_cast<const float *>(a.uy);
  const float *uzs = static_cast<const float *>(a.uz);
  for (;;) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(aa.tile_counter, 1u);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= total) break;
    int lo = 0, hi = aa.n_sets;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (s_prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    const int set = lo;
    if (set != s_set) {
      const int words = (int)(sizeof(Pulse<float>) / 4);
      const uint32_t *src = reinterpret_cast<const uint32_t *>(sets + set);
      uint32_t *dst = reinterpret_cast<uint32_t *>(s_pulse_raw);
      for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0) s_set = set;
    }
    __syncthreads();
    const long long off0 = aa.set_offsets ? aa.set_offsets[set] : 0;
    const long long off1 = aa.set_offsets ? aa.set_offsets[set + 1] : a.n;
    const long long i0 = off0 + (tile - s_prefix[set]) * kPer + threadIdx.x;
    const long long i1 = i0 + kAdjBlock;
    const bool v0 = i0 >= 0 && i0 < off1 && i0 < a.n;
    const bool v1 = i1 >= 0 && i1 < off1 && i1 < a.n;
    const double Ns = (double)(off1 - off0);
    // ---- forward pass with checkpoints
    double X[2] = {0.0, 0.0}, Y[2] = {0.0, 0.0}, Z[2] = {0.0, 0.0};
    float ua[3] = {0.0f, 0.0f, 0.0f}, ub[3] = {0.0f, 0.0f, 0.0f};
    if (v0) {
      X[0] = a.x[i0]; Y[0] = a.y[i0]; Z[0] = a.z[i0];
      ua[0] = uxs[i0]; ua[1] = uys[i0]; ua[2] = uzs[i0];
    }
    if (v1) {
      X[1] = a.x[i1]; Y[1] = a.y[i1]; Z[1] = a.z[i1];
      ub[0] = uxs[i1]; ub[1] = uys[i1]; ub[2] = uzs[i1];
    }
    Pos2 pos;
    pos.load(X, Y, Z, P.z_f);
    F2 u[3] = {F2(ua[0], ub[0]), F2(ua[1], ub[1]), F2(ua[2], ub[2])};
    TimeBase<AP_FP32_PHASEFF> tb;
    tb.init(P, a.t0, a.dt);
    const float dts = (float)a.dt;
    const F2 dtR = dts, dtxy = dts * P.adv_xy;
    for (int seg = 0; seg < aa.n_seg; ++seg) {
      const long long s0 = (long long)seg * aa.K;
      const int cnt = (int)(a.n_steps - s0 < aa.K ? a.n_steps - s0 : aa.K);
      PairIO::put(ck + (size_t)seg * PairIO::W * stride, stride, pos, u);
      __syncthreads();
      for (int k = threadIdx.x; k < cnt; k += blockDim.x) s_steps[k] = tb.at(s0 + k);
      __syncthreads();
      for (int k = 0; k < cnt; ++k) {
        const Local<F2> L = local_coords2(P, s_steps[k], pos);
        F2 E[3], B[3];
        analytic_fields<KIND, AP_FP32_PHASEFF, F2>(P, L, E, B);
        const F2 ig = boris(u, E, B, dtR);
        pos.advance(u[0] * ig, u[1] * ig, u[2] * ig, dtxy, dtR);
      }
    }
    // ---- objective and seed, per particle
    const float uf[2][3] = {{u[0].x, u[1].x, u[2].x}, {u[0].y, u[1].y, u[2].y}};
    double gN[2], Jv = 0.0;
    float sd[2][3];
    for (int h = 0; h < 2; ++h) {
      const bool vh = h ? v1 : v0;
      gN[h] = sqrt(1.0 + (double)uf[h][0] * uf[h][0] + (double)uf[h][1] * uf[h][1] +
                   (double)uf[h][2] * uf[h][2]);
      for (int k = 0; k < 3; ++k) sd[h][k] = vh ? (float)((double)uf[h][k] / (gN[h] * Ns)) : 0.0f;
      if (vh) Jv += gN[h] / Ns;
    }
    F2 lx[3] = {F2(0.0f), F2(0.0f), F2(0.0f)};
    F2 lu[3] = {F2(sd[0][0], sd[1][0]), F2(sd[0][1], sd[1][1]), F2(sd[0][2], sd[1][2])};
    double gacc[kNp] = {0.0, 0.0, 0.0, 0.0};
    // ---- reverse sweep over segments
    for (int seg = aa.n_seg - 1; seg >= 0; --seg) {
      const long long s0 = (long long)seg * aa.K;
      const int cnt = (int)(a.n_steps - s0 < aa.K ? a.n_steps - s0 : aa.K);
      PairIO::get(ck + (size_t)seg * PairIO::W * stride, stride, pos, u);
      __syncthreads();
      for (int k = threadIdx.x; k < cnt; k += blockDim.x) s_steps[k] = tb.at(s0 + k);
      __syncthreads();
      for (int k = 0; k < cnt; ++k) {
        PairIO::put(tp + (size_t)k * PairIO::W * stride, stride, pos, u);
        const Local<F2> L = local_coords2(P, s_steps[k], pos);
        F2 E[3], B[3];
        analytic_fields<KIND, AP_FP32_PHASEFF, F2>(P, L, E, B);
        const F2 ig = boris(u, E, B, dtR);
        pos.advance(u[0] * ig, u[1] * ig, u[2] * ig, dtxy, dtR);
      }
      // the tape entries this thread just stored are read back by its own
      // asynchronous copies
      __threadfence_block();
      auto stage = [&](int k) {
        const float2 *src = tp + (size_t)k * PairIO::W * stride;
#pragma unroll
        for (int w = 0; w < PairIO::W; ++w)
          cp_async8((unsigned)__cvta_generic_to_shared(s_next + ((k & 1) * PairIO::W + w) * kAdjBlock +
                                                       threadIdx.x),
                    src + (size_t)w * stride);
      };
      F2 gs[kNp] = {F2(0.0f), F2(0.0f), F2(0.0f), F2(0.0f)};
      stage(cnt - 1);
      for (int k = cnt - 1; k >= 0; --k) {
        cp_async_wait_all();
        PairIO::get(s_next + (k & 1) * PairIO::W * kAdjBlock + threadIdx.x, kAdjBlock, pos, u);
        if (k > 0) stage(k - 1);
        reverse_step_pair<KIND>(P, dts, s_steps[k], pos, u, lx, lu, gs);
      }
      for (int k = 0; k < kNp; ++k)
        gacc[k] += (v0 ? (double)gs[k].x : 0.0) + (v1 ? (double)gs[k].y : 0.0);
    }
    if ((v0 || v1) && !(isfinite(gacc[0]) && isfinite(gacc[1]) && isfinite(gacc[2]) && isfinite(gacc[3])))
      atomicOr(a.status, kStatusNonfinite);
    // per-set reduction (every particle of the tile belongs to `set`)
    for (int k = 0; k < kNp; ++k) {
      double t = block_sum(gacc[k], s_red);
      if (threadIdx.x == 0) atomicAdd(aa.dJ + (size_t)set * AP_NPARAM + k, t);
    }
    if (aa.J) {
      double t = block_sum(Jv, s_red);
      if (threadIdx.x == 0) atomicAdd(aa.J + set, t);
    }
    __syncthreads();
  }
}

template <int KIND>
int launch_adjoint_pair(const Pulse<float> *sets, const AdjArgs &aa, void *stream) {
  auto kern = adjoint_kernel_pair<KIND>;
  const size_t dyn = 2 * (size_t)PairIO::W * kAdjBlock * sizeof(float2);
  // static (about 40 KB) plus dynamic shared memory passes 48 KB: opt in
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
    return AP_ERR_CUDA;
  const int grid = (int)(aa.nslots / (2 * kAdjBlock));
  kern<<<grid, kAdjBlock, dyn, static_cast<cudaStream_t>(stream)>>>(sets, aa);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

template <int KIND, int PREC, bool GRID>
int launch_adjoint_t(const Pulse<Real<PREC>> *sets, const AdjArgs &aa, int grid, void *stream) {
  auto kern = adjoint_kernel<KIND, PREC, GRID>;
  const size_t dyn = 2 * (size_t)StateIO<PREC>::W * kAdjBlock * sizeof(typename StateIO<PREC>::T);
  // static (about 40 KB) plus dynamic shared memory passes 48 KB: opt in
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
    return AP_ERR_CUDA;
  kern<<<grid, kAdjBlock, dyn, static_cast<cudaStream_t>(stream)>>>(sets, aa);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

template <int KIND>
int launch_adjoint_k(int precision, const Pulse<double> *dpd, const Pulse<float> *dpf,
                     const AdjArgs &aa, int grid, void *stream) {
  const bool gr = aa.base.grid_on != 0;
  if (precision == AP_FP64)
    return gr ? launch_adjoint_t<KIND, AP_FP64, true>(dpd, aa, grid, stream)
              : launch_adjoint_t<KIND, AP_FP64, false>(dpd, aa, grid, stream);
  if (precision == AP_FP32_PHASEFF) {
    if constexpr (KIND == AP_GAUSS || KIND == AP_FLYING_CF)
      if (!gr) return launch_adjoint_pair<KIND>(dpf, aa, stream);
    return gr ? launch_adjoint_t<KIND, AP_FP32_PHASEFF, true>(dpf, aa, grid, stream)
              : launch_adjoint_t<KIND, AP_FP32_PHASEFF, false>(dpf, aa, grid, stream);
  }
  return AP_ERR_UNSUPPORTED;
}

}  // namespace apt

// Host side: the handle internals live in ap_api.cu; these accessors expose
// what the adjoint launch needs.
namespace apt {
int handle_info(ap_handle h, int *device, int *sm_count, int *n_sets, int *uniform_kind,
                const Pulse<double> **dpd, const Pulse<float> **dpf, int **status);
int handle_push_args(ap_handle h, const ap_particles *p, const ap_grid *g, double t0, double dt,
                     int64_t n_steps, int32_t precision, PushArgs *a, void *stream);
}  // namespace apt

namespace {
// particle slots of the workspace: the larger of the one-particle kernel's
// (kAdjBlocksPerSm blocks of kAdjBlock per SM) and the two-particle
// kernel's (kAdjPairBlocksPerSm blocks of 2 kAdjBlock particles)
long long adj_slots(int sm_count) {
  const int a = apt::kAdjBlocksPerSm * apt::kAdjBlock, b = apt::kAdjPairBlocksPerSm * 2 * apt::kAdjBlock;
  return (long long)sm_count * (a > b ? a : b);
}
}  // namespace

extern "C" {

size_t ap_adjoint_workspace_bytes(ap_handle h, int64_t n, int64_t n_steps, int32_t ckpt_every) {
  int dev, sm, ns, uk, *st;
  const apt::Pulse<double> *pd;
  const apt::Pulse<float> *pf;
  if (!h || n < 0 || n_steps < 1 || ckpt_every < 1 || ckpt_every > apt::kAdjMaxK) return 0;
  if (apt::handle_info(h, &dev, &sm, &ns, &uk, &pd, &pf, &st) != AP_OK) return 0;
  const long long slots = adj_slots(sm);
  const long long n_seg = (n_steps + ckpt_every - 1) / ckpt_every;
  return 256 + (size_t)(n_seg + ckpt_every) * apt::kAdjStateBytes * (size_t)slots;
}

int ap_push_adjoint(ap_handle h, const ap_particles *p0, const ap_grid *g, double t0, double dt,
                    int64_t n_steps, int32_t ckpt_every, int32_t objective, int32_t precision,
                    double *dJ_dparams, double *J_out, void *workspace, size_t ws_bytes,
                    void *stream) {
  int dev, sm, ns, uk, *status;
  const apt::Pulse<double> *dpd;
  const apt::Pulse<float> *dpf;
  if (!h || !p0 || !dJ_dparams) return AP_ERR_ARG;
  int rc = apt::handle_info(h, &dev, &sm, &ns, &uk, &dpd, &dpf, &status);
  if (rc != AP_OK) return rc;
  if (objective != AP_OBJ_MEAN_GAMMA) return AP_ERR_ARG;
  if (precision != AP_FP64 && precision != AP_FP32_PHASEFF) return AP_ERR_UNSUPPORTED;
  if (uk < 0 || uk == AP_FLYING_SUM) return AP_ERR_UNSUPPORTED;
  if (n_steps < 1 || ckpt_every < 1 || ckpt_every > apt::kAdjMaxK) return AP_ERR_ARG;
  if (p0->set_offsets ? p0->n_sets != ns : ns != 1) return AP_ERR_ARG;
  const size_t need = ap_adjoint_workspace_bytes(h, p0->n, n_steps, ckpt_every);
  if (!workspace || ws_bytes < need) return AP_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return AP_ERR_ALIGN;
  apt::AdjArgs aa;
  std::memset(&aa, 0, sizeof(aa));
  rc = apt::handle_push_args(h, p0, g, t0, dt, n_steps, precision, &aa.base, stream);
  if (rc != AP_OK) return rc;
  if (aa.base.grid.cells) {
    rc = apt::drop_cell_layout(aa.base.grid);
    if (rc != AP_OK) return rc;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(dJ_dparams, 0, sizeof(double) * AP_NPARAM * ns, s) != cudaSuccess ||
      (J_out && cudaMemsetAsync(J_out, 0, sizeof(double) * ns, s) != cudaSuccess) ||
      cudaMemsetAsync(workspace, 0, 256, s) != cudaSuccess)
    return AP_ERR_CUDA;
  if (p0->n == 0) return AP_OK;
  const long long slots = adj_slots(sm);
  const long long n_seg = (n_steps + ckpt_every - 1) / ckpt_every;
  char *ws = static_cast<char *>(workspace);
  const size_t w = (precision == AP_FP64) ? sizeof(double) * 6 : sizeof(float) * 9;
  aa.set_offsets = reinterpret_cast<const long long *>(p0->set_offsets);
  aa.n_sets = ns;
  aa.K = ckpt_every;
  aa.n_seg = (int)n_seg;
  aa.tile_counter = reinterpret_cast<unsigned int *>(ws);
  aa.ckpt = ws + 256;
  aa.tape = ws + 256 + (size_t)n_seg * w * slots;
  aa.nslots = slots;
  aa.dJ = dJ_dparams;
  aa.J = J_out;
  const int grid = sm * apt::kAdjBlocksPerSm;  // the one-particle kernel's launch
  switch (uk) {
    case AP_PLANE: return apt::launch_adjoint_k<AP_PLANE>(precision, dpd, dpf, aa, grid, stream);
    case AP_GAUSS: return apt::launch_adjoint_k<AP_GAUSS>(precision, dpd, dpf, aa, grid, stream);
    case AP_LG: return apt::launch_adjoint_k<AP_LG>(precision, dpd, dpf, aa, grid, stream);
    case AP_FLYING_CF:
      return apt::launch_adjoint_k<AP_FLYING_CF>(precision, dpd, dpf, aa, grid, stream);
    default: return AP_ERR_UNSUPPORTED;
  }
}

}  // extern "C"
