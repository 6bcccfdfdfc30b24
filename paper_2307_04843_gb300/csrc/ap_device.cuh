// ap_device.cuh -- device code of the analytic-pulse gather + Boris push.
//
// Everything a particle needs for one step, templated on the arithmetic of
// the push:
//   PREC = AP_FP64          double everywhere (the plain FP64 GPU path);
//   PREC = AP_FP32_PHASE64  float fields and Boris, native double phase and
//                           position accumulation;
//   PREC = AP_FP32_PHASEFF  float fields and Boris, phase and position as
//                           float-float pairs (no FP64 instruction in the
//                           step loop; the FP64 pipe of this GPU issues at
//                           about 1/70 of the FP32 rate).
//
// Method references (arXiv:2307.04843): field split E = E1 + E2 (Sec. 2,
// Eqs. E_1, E_2); plane-wave pulse (Eqs. plane_func, plane_b); paraxial
// Gaussian beam (Eq. paraxial, rewritten for +z and D = 3) in the complex
// beam-parameter form q = 1 / (1 - i zeta); longitudinal components from the
// divergence conditions (Sec. 3.1); flying focus as a linear superposition of
// spectral components (Sec. 3.3).  The Boris step is the textbook relativistic
// scheme (Boris 1970); the paper does not specify a pusher.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>
#include <type_traits>

#include "ap_internal.h"

namespace apt {

template <int PREC>
using Real = typename std::conditional<PREC == AP_FP64, double, float>::type;

// True for the packed pair type of ap_pair.cuh (two particles per value).
template <typename R>
struct IsPair : std::false_type {};

// ------------------------------------------------------------ float-float
// Error-free transformations (Knuth TwoSum, Dekker/FMA TwoProd).  The _rn
// intrinsics keep the compiler from contracting or reassociating them.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ FF two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

// the _rn spellings shared with the packed pair type (templates call these)
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ FF split_double(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(v - (double)hi);
  return {hi, lo};
}

// 2 pi = P1 + P2 (+ ~2e-15): Cody & Waite (1980) two-constant split.
constexpr float kTwoPiHi = 6.28318548202514648f;
constexpr float kTwoPiLo = -1.74845553e-07f;
constexpr float kInvTwoPi = 0.159154943091895336f;

// Round to the nearest integer on the FP32 pipe: adding 1.5 * 2^23 forces
// the unit in the last place to 1 (valid for |x| < 2^22), one FFMA/FADD and
// one FADD instead of a conversion-pipe FRND.
constexpr float kRoundMagic = 12582912.0f;
__device__ __forceinline__ float round_fma(float a, float b) {
  return __fsub_rn(__fmaf_rn(a, b, kRoundMagic), kRoundMagic);
}

// (hi + lo) reduced modulo 2 pi to about [-pi, pi], rounded to float.
// m = rint(hi / 2 pi); hi - m P1 is exact (Sterbenz) with m P1 split by
// TwoProd; the low-order parts are summed in float.
__device__ __forceinline__ float reduce_ff(float hi, float lo) {
  float m = round_fma(hi, kInvTwoPi);
  FF p = two_prod(m, kTwoPiHi);
  float r = __fsub_rn(hi, p.hi);
  float t = __fsub_rn(__fsub_rn(lo, p.lo), __fmul_rn(m, kTwoPiLo));
  return __fadd_rn(r, t);
}

// float argument reduction for moderate |x| (a few times 2 pi).
__device__ __forceinline__ float reduce_f(float x) {
  float m = round_fma(x, kInvTwoPi);
  x = fmaf(-m, kTwoPiHi, x);
  return fmaf(-m, kTwoPiLo, x);
}

// Special-function unit (MUFU) instructions, written as PTX so that each is
// one approximate hardware operation (documented maximum errors: sin/cos
// 2^-20.9 absolute on [-pi, pi], ex2 2^-22.5 relative, rcp 1 ulp, rsqrt
// 2^-22.9 relative); subnormal results flush to zero.
__device__ __forceinline__ float mufu_sin(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_cos(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void sincos_r(float x, float *s, float *c) {
  *s = mufu_sin(x);
  *c = mufu_cos(x);
}
__device__ __forceinline__ void sincos_r(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ float exp2_r(float x) { return mufu_ex2(x); }
__device__ __forceinline__ double exp2_r(double x) { return exp2(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return mufu_rsqrt(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float rcp_r(float x) { return mufu_rcp(x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }
__device__ __forceinline__ float cos_r(float x) { return mufu_cos(x); }
__device__ __forceinline__ double cos_r(double x) { return cos(x); }

template <typename R>
struct Cx {
  R re, im;
};
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> cscale(Cx<R> a, R s) {
  return {a.re * s, a.im * s};
}

constexpr double kLog2e = 1.4426950408889634;

// ------------------------------------------------------------ positions
// Position of one particle in the arithmetic of PREC.
template <int PREC>
struct Pos;

template <>
struct Pos<AP_FP64> {
  double x, y, z;
  __device__ void load(double X, double Y, double Z) { x = X; y = Y; z = Z; }
  __device__ void store(double *X, double *Y, double *Z) const { *X = x; *Y = y; *Z = z; }
  // dt_xy = dt, or 0 for a 1D-3V set
  __device__ void advance(double vx, double vy, double vz, double dt_xy, double dt) {
    x += dt_xy * vx; y += dt_xy * vy; z += dt * vz;
  }
  __device__ double xr() const { return x; }
  __device__ double yr() const { return y; }
  __device__ double zr() const { return z; }
};

template <>
struct Pos<AP_FP32_PHASE64> {
  double x, y, z;
  __device__ void load(double X, double Y, double Z) { x = X; y = Y; z = Z; }
  __device__ void store(double *X, double *Y, double *Z) const { *X = x; *Y = y; *Z = z; }
  // dt u / gamma in float, accumulated in double
  __device__ void advance(float vx, float vy, float vz, float dt_xy, float dt) {
    x += (double)(dt_xy * vx); y += (double)(dt_xy * vy); z += (double)(dt * vz);
  }
  __device__ float xr() const { return (float)x; }
  __device__ float yr() const { return (float)y; }
  __device__ float zr() const { return (float)z; }
};

template <>
struct Pos<AP_FP32_PHASEFF> {
  FF x, y, z;
  __device__ void load(double X, double Y, double Z) {
    x = split_double(X); y = split_double(Y); z = split_double(Z);
  }
  __device__ void store(double *X, double *Y, double *Z) const {
    *X = (double)x.hi + (double)x.lo;
    *Y = (double)y.hi + (double)y.lo;
    *Z = (double)z.hi + (double)z.lo;
  }
  // Compensated (Kahan) accumulation of the float increment: the low part
  // carries the rounding error of every add, so hi + lo is the exact sum of
  // the increments to within O(2^-48) relative (Kahan 1965; the error term
  // is exact whenever |hi| >= |increment|, the normal case).
  __device__ __forceinline__ static void acc(FF &p, float d) {
    float y = __fadd_rn(d, p.lo);
    float t = __fadd_rn(p.hi, y);
    p.lo = __fsub_rn(y, __fsub_rn(t, p.hi));
    p.hi = t;
  }
  // a zero increment (1D-3V) leaves a normalised pair unchanged
  __device__ void advance(float vx, float vy, float vz, float dt_xy, float dt) {
    acc(x, __fmul_rn(dt_xy, vx)); acc(y, __fmul_rn(dt_xy, vy)); acc(z, __fmul_rn(dt, vz));
  }
  __device__ float xr() const { return __fadd_rn(x.hi, x.lo); }
  __device__ float yr() const { return __fadd_rn(y.hi, y.lo); }
  __device__ float zr() const { return __fadd_rn(z.hi, z.lo); }
};

// ------------------------------------------------------------ time base
// Per-thread constants of the time stepping, made once from (t0, dt) in
// double: t_n = t0 + n dt is recomputed for every step, never accumulated.
// `at(n)` gives the per-step value: t_n in double for the double-phase
// variants; for the float-float variant the reduced carrier phase
// C_n = omega (t_n - t_f) + phase0 (mod 2 pi) and T_n = t_n - t_f as a
// float-float pair, which the kernels tabulate once per block in shared
// memory (every particle of a block shares them).
struct StepFF {
  float C, Th, Tl, pad;
};

template <int PREC>
struct TimeBase;

template <>
struct TimeBase<AP_FP64> {
  using Step = double;
  double t0, dt;
  template <typename P>
  __device__ void init(const P &, double T0, double DT) { t0 = T0; dt = DT; }
  __device__ double at(long long n) const { return t0 + (double)n * dt; }
};
template <>
struct TimeBase<AP_FP32_PHASE64> {
  using Step = double;
  double t0, dt;
  template <typename P>
  __device__ void init(const P &, double T0, double DT) { t0 = T0; dt = DT; }
  __device__ double at(long long n) const { return t0 + (double)n * dt; }
};
template <>
struct TimeBase<AP_FP32_PHASEFF> {
  using Step = StepFF;
  // C_n = Om0 + n Del (mod 2 pi), Om0 and Del reduced in double on entry;
  // T_n = T0 + n DT.
  FF om0, del, T0, DT;
  template <typename P>
  __device__ void init(const P &pp, double t0, double dt) {
    const double twopi = 2.0 * CUDART_PI;
    double c0 = pp.omega * (t0 - pp.t_f) + pp.phase0;
    c0 -= twopi * rint(c0 / twopi);
    double d = pp.omega * dt;
    d -= twopi * rint(d / twopi);
    om0 = split_double(c0);
    del = split_double(d);
    T0 = split_double(t0 - pp.t_f);
    DT = split_double(dt);
  }
  __device__ StepFF at(long long n) const { return at_f((float)n); }  // exact for n < 2^24
  // the same with the level given as a float holding an integer below 2^24
  // (callers that count in float avoid the int-to-float conversion)
  __device__ StepFF at_f(float nf) const {
    FF nd = two_prod(nf, del.hi);
    FF c = two_sum(om0.hi, nd.hi);
    float clo = __fadd_rn(__fadd_rn(c.lo, nd.lo), __fmaf_rn(nf, del.lo, om0.lo));
    FF nt = two_prod(nf, DT.hi);
    FF T = two_sum(T0.hi, nt.hi);
    T.lo = __fadd_rn(T.lo, __fadd_rn(nt.lo, __fmaf_rn(nf, DT.lo, T0.lo)));
    return {reduce_ff(c.hi, clo), T.hi, T.lo, 0.0f};
  }
};

// Local coordinates of one particle at one step, relative to the focus:
// transverse x, y; dz = z - z_f; the reduced carrier phase psi; envelope
// argument eta = (t - t_f) - (z - z_f)/v_g; and for the flying focus the
// light-front coordinate phi' = (t - t_f) - (z - z_f) split in two parts.
template <typename R>
struct Local {
  R x, y, dz, psi, eta;
  R T;              // t - t_f (closed-form flying focus)
  R phi_hi, phi_lo;  // flying focus only (float-float, or double in phi_hi)
};

template <int PREC>
__device__ __forceinline__ Local<Real<PREC>> local_coords(const Pulse<Real<PREC>> &P,
                                                          const typename TimeBase<PREC>::Step &st,
                                                          const Pos<PREC> &pos) {
  Local<Real<PREC>> L;
  if constexpr (PREC == AP_FP64) {
    double T = st - P.t_f;
    double dz = pos.z - P.z_f;
    L.x = pos.x;
    L.y = pos.y;
    L.dz = dz;
    L.psi = P.omega * T - P.k * dz + P.phase0;
    L.eta = T - dz * P.inv_vg;
    L.T = T;
    L.phi_hi = T - dz;
    L.phi_lo = 0.0;
  } else if constexpr (PREC == AP_FP32_PHASE64) {
    double T = st - P.t_f;
    double dz = pos.z - P.z_f;
    double psi = P.omega * T - P.k * dz + P.phase0;
    const double twopi = 2.0 * CUDART_PI;
    psi = fma(-rint(psi * (1.0 / twopi)), twopi, psi);
    L.x = (float)pos.x;
    L.y = (float)pos.y;
    L.dz = (float)dz;
    L.psi = (float)psi;
    L.eta = (float)(T - dz * (double)P.inv_vg);
    L.T = (float)T;
    double phi = T - dz;
    L.phi_hi = (float)phi;
    L.phi_lo = (float)(phi - (double)L.phi_hi);
  } else {
    // dz = z - z_f
    FF dz = two_sum(pos.z.hi, -P.zf_hi);
    dz.lo = __fadd_rn(dz.lo, __fsub_rn(pos.z.lo, P.zf_lo));
    // psi = C_n - k dz
    FF kd = two_prod(P.k_hi, dz.hi);
    kd.lo = __fadd_rn(kd.lo, __fmaf_rn(P.k_hi, dz.lo, __fmul_rn(P.k_lo, dz.hi)));
    FF ps = two_sum(st.C, -kd.hi);
    L.psi = reduce_ff(ps.hi, __fsub_rn(ps.lo, kd.lo));
    L.x = pos.xr();
    L.y = pos.yr();
    L.dz = __fadd_rn(dz.hi, dz.lo);
    float Tf = __fadd_rn(st.Th, st.Tl);
    L.eta = fmaf(-L.dz, P.inv_vg, Tf);
    L.T = Tf;
    // phi' = T - dz as float-float
    FF ph = two_sum(st.Th, -dz.hi);
    L.phi_hi = ph.hi;
    L.phi_lo = __fadd_rn(ph.lo, __fsub_rn(st.Tl, dz.lo));
  }
  return L;
}

// ------------------------------------------------------------ envelope
// Gamma(eta) split into a multiplicative factor `mul` and an additive
// base-2 exponent `l2` (Gaussian and super-Gaussian envelopes share the
// beam's exp2).  SIN2: env_a = pi/T, env_b = T/2; GAUSS: env_a = 2 ln2 log2e
// / T^2; SGAUSS: env_a = 1/tau, env_b = log2e; CW: 1.
template <class PT, typename R>
__device__ __forceinline__ void envelope(const PT &P, R eta, R &mul, R &l2) {
  mul = R(1);
  l2 = R(0);
  switch (P.env) {
    case AP_ENV_SIN2: {
      if constexpr (IsPair<R>::value) {
        // both halves evaluated, each cleared outside its own window
        const R c = cos_r(eta * P.env_a);
        mul = sin2_window(c * c, eta, P.env_b);
      } else if (fabs(eta) > P.env_b) {
        mul = R(0);
      } else {
        R c = cos_r(eta * P.env_a);
        mul = c * c;
      }
      break;
    }
    case AP_ENV_GAUSS:
      l2 = -P.env_a * eta * eta;
      break;
    case AP_ENV_SGAUSS: {
      R s = eta * P.env_a;
      s = s * s;
      R p = s;
      for (int i = 1; i < P.sg_order; ++i) p *= s;
      l2 = -P.env_b * p;
      break;
    }
    default:
      break;
  }
}

// --------------------------------------------------------- field assembly
// E_perp = Re[p U], B_perp = (B0/E0) Re[(z x p) U];
// E_z = Re[-i (v_phi/omega) DE], B_z = (B0/E0) Re[-i (c/omega) DB] with
// DE = p_x dU/dx + p_y dU/dy and DB = -p_y dU/dx + p_x dU/dy (Sec. 3.1).
template <class PT, typename R>
__device__ __forceinline__ void assemble(const PT &P, Cx<R> U, Cx<R> DE, Cx<R> DB, bool lon,
                                         R E[3], R B[3]) {
  R pxU = P.px_re * U.re - P.px_im * U.im;
  R pyU = P.py_re * U.re - P.py_im * U.im;
  E[0] = pxU;
  E[1] = pyU;
  B[0] = -P.bratio * pyU;
  B[1] = P.bratio * pxU;
  if (lon) {
    E[2] = P.lonE * DE.im;
    B[2] = P.bratio * P.lonB * DB.im;
  } else {
    E[2] = R(0);
    B[2] = R(0);
  }
}

// Field assembly for beams whose transverse derivative is
// dU/dx = g x W, dU/dy = g y W (Gaussian: g = -2/w0^2, W = q U; the flying
// focus sums W over components with the 1/k_j factors inside), specialised
// per polarisation (a uniform branch): DE = g (p_x x + p_y y) W and
// DB = g (-p_y x + p_x y) W, E_z = (v_phi/omega) Im DE, B_z = (B0/E0)(c/omega) Im DB.
// finish_beam_pol takes the polarisation as a compile-time parameter, for
// code that assembles several field sets per step and selects it once.
template <int POL, class PT, typename R>
__device__ __forceinline__ void finish_beam_pol(const PT &P, R x, R y, Cx<R> U, Cx<R> W, R g,
                                                bool lon, R E[3], R B[3]) {
  const R br = P.bratio;
  const R ce = P.lonE * g, cb = br * P.lonB * g;
  E[2] = R(0);
  B[2] = R(0);
  if constexpr (POL == AP_LIN_X) {
    E[0] = U.re; E[1] = R(0); B[0] = R(0); B[1] = br * U.re;
    if (lon) { E[2] = ce * x * W.im; B[2] = cb * y * W.im; }
  } else if constexpr (POL == AP_LIN_Y) {
    E[0] = R(0); E[1] = U.re; B[0] = -br * U.re; B[1] = R(0);
    if (lon) { E[2] = ce * y * W.im; B[2] = -cb * x * W.im; }
  } else if constexpr (POL == AP_CIRC_P) {  // p = (1, -i)
    E[0] = U.re; E[1] = U.im; B[0] = -br * U.im; B[1] = br * U.re;
    if (lon) { E[2] = ce * (x * W.im - y * W.re); B[2] = cb * (x * W.re + y * W.im); }
  } else {  // AP_CIRC_M, p = (1, +i)
    E[0] = U.re; E[1] = -U.im; B[0] = br * U.im; B[1] = br * U.re;
    if (lon) { E[2] = ce * (x * W.im + y * W.re); B[2] = cb * (y * W.im - x * W.re); }
  }
}

template <class PT, typename R>
__device__ __forceinline__ void finish_beam(const PT &P, R x, R y, Cx<R> U, Cx<R> W, R g,
                                            bool lon, R E[3], R B[3]) {
  switch (P.pol) {
    case AP_LIN_X: finish_beam_pol<AP_LIN_X>(P, x, y, U, W, g, lon, E, B); break;
    case AP_LIN_Y: finish_beam_pol<AP_LIN_Y>(P, x, y, U, W, g, lon, E, B); break;
    case AP_CIRC_P: finish_beam_pol<AP_CIRC_P>(P, x, y, U, W, g, lon, E, B); break;
    default: finish_beam_pol<AP_CIRC_M>(P, x, y, U, W, g, lon, E, B); break;
  }
}

template <typename R>
__device__ __forceinline__ R reduce_angle(R a) {
  if constexpr (std::is_same<R, float>::value || IsPair<R>::value) return reduce_f(a);
  else return a;
}

// Logarithmic derivatives L1 = Gamma'/Gamma and L2 = Gamma''/Gamma of the
// envelope (the finite-duration terms of Sec. 4).  GAUSS: ln Gamma =
// -2 ln2 eta^2/T^2, so L1 = -lg_c1 eta and L2 = L1^2 - lg_c2 with
// lg_c1 = lg_c2 = 4 ln2/T^2.  SGAUSS: ln Gamma = -u^(2g), u = eta/tau, so with
// q = u^(2g-2): L1 = -lg_c1 u q, L2 = L1^2 - lg_c2 q, lg_c1 = 2g/tau,
// lg_c2 = 2g(2g-1)/tau^2.  CW: zero.
template <class PT, typename R>
__device__ __forceinline__ void envelope_logd(const PT &P, R eta, R &L1, R &L2) {
  L1 = R(0);
  L2 = R(0);
  if (P.env == AP_ENV_GAUSS) {
    L1 = -P.lg_c1 * eta;
    L2 = L1 * L1 - P.lg_c2;
  } else if (P.env == AP_ENV_SGAUSS) {
    const R u = eta * P.env_a;
    const R s = u * u;
    R q = R(1);
    for (int i = 1; i < P.sg_order; ++i) q *= s;
    L1 = -P.lg_c1 * u * q;
    L2 = L1 * L1 - P.lg_c2 * q;
  }
}

// Amplitude factor and phase shift of the lowest finite-duration terms,
// A = 1 - w L2/omega^2 + th^2/2, th = w L1/omega (Eqs. j1 and b_corr_t with
// Phi = 0; w = 1 for J1, w = 1 - v_phi/v_g for B), applied to U as
// A U e^{i th}.
template <typename R, typename S>
__device__ __forceinline__ Cx<R> finite_duration(Cx<R> U, S w, R L1, R L2, S inv_w) {
  const R th = w * L1 * inv_w;
  const R A = R(1) - w * L2 * inv_w * inv_w + R(0.5) * th * th;
  R s, c;
  sincos_r(th, &s, &c);
  return {A * (U.re * c - U.im * s), A * (U.re * s + U.im * c)};
}

// Plane wave (Eqs. plane_func, plane_b): U = A Gamma e^{i psi}.  In a
// plasma (Sec. 4) B is built from U with the finite-duration terms of
// Eq. b_corr_t.
template <class PT, typename R>
__device__ __forceinline__ void fields_plane(const PT &P, const Local<R> &L, R E[3], R B[3]) {
  R mul, l2;
  envelope(P, L.eta, mul, l2);
  R a = P.amp * mul;
  if (l2 != R(0)) a *= exp2_r(l2);
  R s, c;
  sincos_r(L.psi, &s, &c);
  Cx<R> U{a * c, a * s};
  finish_beam(P, L.x, L.y, U, U, R(0), false, E, B);
  if constexpr (PT::kHasPlasma) {
    if (P.plasma) {
      R L1, L2, Et[3];
      envelope_logd(P, L.eta, L1, L2);
      const Cx<R> UB = finite_duration(U, P.fdc, L1, L2, P.inv_w);
      finish_beam(P, L.x, L.y, UB, UB, R(0), false, Et, B);
    }
  }
}

// Analytic current J1 of a plane wave in a linear plasma (Sec. 4, Eq. j1
// with Phi = 0): J = Re[-i (omega_p^2 zeta/omega) A U e^{i th} p],
// th = L1/omega, A = 1 - L2/omega^2 + th^2/2.  J stands for 4 pi J / c.
template <typename R>
__device__ __forceinline__ void current_plane(const Pulse<R> &P, const Local<R> &L, R J[3]) {
  R mul, l2;
  envelope(P, L.eta, mul, l2);
  R a = P.jamp * P.amp * mul;
  if (l2 != R(0)) a *= exp2_r(l2);
  R s, c;
  sincos_r(L.psi, &s, &c);
  R L1, L2;
  envelope_logd(P, L.eta, L1, L2);
  const Cx<R> V = finite_duration(Cx<R>{a * c, a * s}, R(1), L1, L2, R(P.inv_w));
  // Re[p (-i V)] with -i V = (V.im, -V.re)
  J[0] = P.px_re * V.im + P.px_im * V.re;
  J[1] = P.py_re * V.im + P.py_im * V.re;
  J[2] = R(0);
}

// Paraxial Gaussian beam (Eq. paraxial, D = 3, +z):
//   u = A q exp(-r^2 q / w0^2),  q = 1/(1 - i zeta),  zeta = (z - z_f)/z_R,
// which equals A (w0/w) e^{-r^2/w^2} e^{-i k r^2/(2R)} e^{i atan zeta}.
// du/dx = -2 x q / w0^2 u.
// MOVING: closed-form flying focus (Sec. 3.3): the same profile with
// x_f - x -> xi0 - xi, i.e. zeta = ((z - z_f) - beta_f (t - t_f)) / z_R',
// z_R' = (1 - beta_f) z_R (inv_zR holds 1/z_R').
// The Gaussian beam in two parts: what depends on z and t only (the
// envelope, q and the carrier phase), which the grid-node kernels compute
// once per z level and share along a row of nodes, and the transverse part.
template <typename R>
struct BeamZ {
  Cx<R> q;     // 1 / (1 - i zeta)
  R amp_mul;   // A times the envelope's multiplicative factor
  R l2;        // the envelope's base-2 exponent
  R psi;       // reduced carrier phase
};

template <bool MOVING = false, class PT, typename R>
__device__ __forceinline__ BeamZ<R> gauss_z(const PT &P, const Local<R> &L) {
  R mul, l2;
  envelope(P, L.eta, mul, l2);
  R zeta;
  if constexpr (MOVING) zeta = fma(-P.beta_f, L.T, L.dz) * P.inv_zR;
  else zeta = L.dz * P.inv_zR;
  R inv = rcp_r(fma(zeta, zeta, R(1)));
  return {Cx<R>{inv, zeta * inv}, P.amp * mul, l2, L.psi};
}

template <class PT, typename R>
__device__ __forceinline__ void gauss_xy(const PT &P, const BeamZ<R> &Z, R x, R y, R E[3], R B[3]) {
  const Cx<R> q = Z.q;
  R a = (x * x + y * y) * P.inv_w0sq;
  R mag = Z.amp_mul * exp2_r(fma(a * q.re, R(-kLog2e), Z.l2));
  R ang = reduce_angle<R>(Z.psi - a * q.im);
  R s, c;
  sincos_r(ang, &s, &c);
  Cx<R> U = cmul(q, Cx<R>{mag * c, mag * s});
  finish_beam(P, x, y, U, cmul(q, U), R(-2) * P.inv_w0sq, P.lon != 0, E, B);
}

template <bool MOVING = false, class PT, typename R>
__device__ __forceinline__ void fields_gauss(const PT &P, const Local<R> &L, R E[3], R B[3]) {
  gauss_xy(P, gauss_z<MOVING>(P, L), L.x, L.y, E, B);
}

// Laguerre-Gaussian LG_pl (textbook; the paper names the family in Sec. 3.1):
//   u = A (sqrt2/w0)^{|l|} (x + i sgn(l) y)^{|l|} L_p^{|l|}(s) q^{|l|+1} (q/q*)^p e^{-r^2 q/w0^2},
// s = 2 r^2 |q|^2 / w0^2; the longitudinal terms use the product rule.
template <class PT, typename R>
__device__ __forceinline__ void fields_lg(const PT &P, const Local<R> &L, R E[3], R B[3]) {
  R mul, l2;
  envelope(P, L.eta, mul, l2);
  R zeta = L.dz * P.inv_zR;
  R inv = rcp_r(fma(zeta, zeta, R(1)));
  Cx<R> q{inv, zeta * inv};
  R a = (L.x * L.x + L.y * L.y) * P.inv_w0sq;
  R s = R(2) * a * q.re;
  // Two loops with run-time trip counts instead of five (each iteration of a
  // loop costs a branch and its bookkeeping every step):
  // over k < p: L_p^{|l|}(s) and dL/ds = -L_{p-1}^{|l|+1}(s) by the
  // three-term recurrence (accurate where the monomial sum cancels: large s,
  // large p), and g^p with g = q/q*;
  // over i < |l|: (x + i sgn y)^{|l|}, its (|l| - 1)th power, and q^{|l|+1}.
  Cx<R> g{(R(1) - zeta * zeta) * inv, R(2) * zeta * inv};
  R Lp = R(1), Lm = R(0), Dp = R(1), Dm = R(0);
  Cx<R> gp{R(1), R(0)};
  for (int k = 0; k < P.lg_p; ++k) {
    const R Ln = fma(fma(-P.lg_r[1][k], s, P.lg_r[0][k]), Lp, -P.lg_r[2][k] * Lm);
    Lm = Lp;
    Lp = Ln;
    if (k + 1 < P.lg_p) {
      const R Dn = fma(fma(-P.lg_r[4][k], s, P.lg_r[3][k]), Dp, -P.lg_r[5][k] * Dm);
      Dm = Dp;
      Dp = Dn;
    }
    gp = cmul(gp, g);
  }
  const R dL = P.lg_p > 0 ? -Dp : R(0);
  Cx<R> xi{L.x, P.lg_sgn >= 0 ? L.y : -L.y};
  Cx<R> pw{R(1), R(0)}, pwm{R(1), R(0)}, qp = q;
  for (int i = 0; i < P.lg_al; ++i) {
    pwm = pw;
    pw = cmul(pw, xi);
    qp = cmul(qp, q);
  }
  // K = A pref q^{|l|+1} (q/q*)^p
  const Cx<R> K = cscale(cmul(qp, gp), P.amp * P.lg_pref);
  R mag = mul * exp2_r(fma(a * q.re, R(-kLog2e), l2));
  R ang = reduce_angle<R>(L.psi - a * q.im);
  R sn, cs;
  sincos_r(ang, &sn, &cs);
  Cx<R> base = cmul(K, Cx<R>{mag * cs, mag * sn});
  Cx<R> U = cmul(base, cscale(pw, Lp));
  Cx<R> DE{R(0), R(0)}, DB{R(0), R(0)};
  if (P.lon) {
    // dU/dx = base (T1 + x T2), dU/dy = base (i sgn T1 + y T2)
    Cx<R> T1 = cscale(pwm, P.lg_alf * Lp);
    Cx<R> T2 = cmul(pw, Cx<R>{R(4) * q.re * P.inv_w0sq * dL - R(2) * P.inv_w0sq * Lp * q.re,
                              -R(2) * P.inv_w0sq * Lp * q.im});
    R sg = P.lg_sgn >= 0 ? R(1) : R(-1);
    Cx<R> dx = cmul(base, Cx<R>{T1.re + L.x * T2.re, T1.im + L.x * T2.im});
    Cx<R> dy = cmul(base, Cx<R>{-sg * T1.im + L.y * T2.re, sg * T1.re + L.y * T2.im});
    Cx<R> px{P.px_re, P.px_im}, py{P.py_re, P.py_im};
    DE = cadd(cmul(px, dx), cmul(py, dy));
    DB = cadd(cmul(Cx<R>{-py.re, -py.im}, dx), cmul(px, dy));
  }
  assemble(P, U, DE, DB, P.lon != 0, E, B);
}

// Flying focus: linear superposition of Gaussian spectral components
// (Sec. 3.3).  omega_j = w_first + j dw, vacuum k_j = omega_j, so
// e^{i omega_j phi'} = e^{i w_first phi'} (e^{i dw phi'})^j: two reduced
// base angles and one complex rotation per component.
template <int PREC, typename R = Real<PREC>>
__device__ __forceinline__ void fields_flying(const Pulse<Real<PREC>> &P, const Local<R> &L,
                                              R E[3], R B[3]) {
  R A1, B1;
  if constexpr (PREC == AP_FP64) {
    A1 = P.ff_w * L.phi_hi;
    B1 = P.ff_dw * L.phi_hi;
  } else {
    // (w_first + 0) * phi' and dw * phi' in float-float, reduced mod 2 pi
    const R whi = P.ffw_hi, wlo = P.ffw_lo, dhi = P.ffd_hi, dlo = P.ffd_lo;
    const auto a = two_prod(whi, L.phi_hi);
    const R alo = fma_rn(whi, L.phi_lo, fma_rn(wlo, L.phi_hi, a.lo));
    A1 = reduce_ff(a.hi, alo);
    const auto b = two_prod(dhi, L.phi_hi);
    const R blo = fma_rn(dhi, L.phi_lo, fma_rn(dlo, L.phi_hi, b.lo));
    B1 = reduce_ff(b.hi, blo);
  }
  R sa, ca, sb, cb;
  sincos_r(A1, &sa, &ca);
  sincos_r(B1, &sb, &cb);
  Cx<R> rot{ca, sa};
  const Cx<R> step{cb, sb};
  const R a = (L.x * L.x + L.y * L.y) * P.inv_w0sq;
  const R ak = -a * R(kLog2e);
  Cx<R> S0{R(0), R(0)}, S1{R(0), R(0)};
  const int nc = P.n_comp;
  for (int j = 0; j < nc; ++j) {
    const auto &cj = P.comp[j];
    R zeta = fma(L.dz, cj.inv_zR, -cj.zoff);
    R inv = rcp_r(fma(zeta, zeta, R(1)));
    Cx<R> q{inv, zeta * inv};
    R mag = exp2_r(ak * q.re);
    R s, c;
    sincos_r(-a * q.im, &s, &c);
    Cx<R> U = cmul(cmul(q, Cx<R>{mag * c, mag * s}), cmul(rot, Cx<R>{cj.c_re, cj.c_im}));
    S0 = cadd(S0, U);
    if (P.lon) S1 = cadd(S1, cscale(cmul(q, U), cj.inv_k));
    rot = cmul(rot, step);
  }
  // the 1/k_j factors are inside S1: lonE = lonB = 1 for this kind
  finish_beam(P, L.x, L.y, S0, S1, R(-2) * P.inv_w0sq, P.lon != 0, E, B);
}

// R is Real<PREC>, or for the two-particle float-float kernels the packed
// pair type of ap_pair.cuh.
template <int KIND, int PREC, typename R = Real<PREC>>
__device__ __forceinline__ void analytic_fields(const Pulse<Real<PREC>> &P, const Local<R> &L,
                                                R E[3], R B[3]) {
  if constexpr (KIND == AP_PLANE) fields_plane(P, L, E, B);
  else if constexpr (KIND == AP_GAUSS) fields_gauss(P, L, E, B);
  else if constexpr (KIND == AP_LG) fields_lg(P, L, E, B);
  else if constexpr (KIND == AP_FLYING_CF) fields_gauss<true>(P, L, E, B);
  else fields_flying<PREC, R>(P, L, E, B);
}

// ------------------------------------------------------------ grid gather
// Trilinear gather of the static node-centred grid (E = E1 + E2, Sec. 2).
// Because the grid is static, the 8 corner values of the particle's current
// cell are kept in registers as trilinear coefficients and refetched only
// when the particle changes cell; the result equals a gather every step.
template <typename R>
struct GridCache {
  R ox, oy, oz;  // lower corner of the cached cell in grid units (-16: nothing cached)
  R wx, wy, wz;  // trilinear weights of the current step
  R c[6][8];     // raw corner values c[comp][cx + 2 cy + 4 cz] of the cached cell
};

template <typename R>
__device__ __forceinline__ void grid_cache_reset(GridCache<R> &gc) {
  gc.ox = gc.oy = gc.oz = R(-16);
}

// position in grid units, clamped to the node range [0, top = n - 1]
template <typename R>
__device__ __forceinline__ R grid_unit(R v, R inv_d, R off, R top) {
  return fmin(fmax(fma(v, inv_d, off), R(0)), top);
}

// Phase 1 of the gather, called at the start of a step: the particle's
// weights in its cell; on a cell change the corner values of the new cell
// are requested into the cache (raw), so that their memory latency overlaps
// the analytic field evaluation that runs before grid_eval.
template <typename R>
__device__ __forceinline__ void grid_fetch(const GridView &g, GridCache<R> &gc, R x, R y, R z) {
  R fx, fy, fz;
  if constexpr (std::is_same<R, double>::value) {
    fx = grid_unit<R>(x, g.inv_d_d[0], g.off_d[0], R(g.nx - 1));
    fy = grid_unit<R>(y, g.inv_d_d[1], g.off_d[1], R(g.ny - 1));
    fz = grid_unit<R>(z, g.inv_d_d[2], g.off_d[2], R(g.nz - 1));
  } else {
    fx = grid_unit<R>(x, g.inv_d[0], g.off[0], R(g.top[0]));
    fy = grid_unit<R>(y, g.inv_d[1], g.off[1], R(g.top[1]));
    fz = grid_unit<R>(z, g.inv_d[2], g.off[2], R(g.top[2]));
  }
  R wx = fx - gc.ox, wy = fy - gc.oy, wz = fz - gc.oz;
  // still inside the cached cell (the upper face included, as for the last
  // cell of the grid): no integer work, no loads.  The warp-uniform test in
  // front keeps the refetch a real branch (taken only when some lane of the
  // warp changed cell) instead of predicated code issued every step; every
  // lane of the warp calls this together.
  const bool need = !(wx >= R(0) && wx <= R(1) && wy >= R(0) && wy <= R(1) && wz >= R(0) && wz <= R(1));
  if (__any_sync(0xffffffffu, need) && need) {
    int ix, iy, iz;
    if constexpr (std::is_same<R, float>::value) {
      // lower cell corner without the conversion pipe: rint(f - 1/2) through
      // the 1.5 * 2^23 magic number (a face point may land in the cell below,
      // where its weight is 1: same value), clamped to [0, n - 2]; the
      // integer is read from the bits of (corner + magic)
      auto corner = [](float f, int n, int &i) {
        float c = __fsub_rn(__fadd_rn(__fsub_rn(f, 0.5f), kRoundMagic), kRoundMagic);
        c = fminf(fmaxf(c, 0.0f), (float)(n - 2));
        i = __float_as_int(__fadd_rn(c, kRoundMagic)) - __float_as_int(kRoundMagic);
        return c;
      };
      gc.ox = corner(fx, g.nx, ix);
      gc.oy = corner(fy, g.ny, iy);
      gc.oz = corner(fz, g.nz, iz);
    } else {
      ix = min((int)fx, g.nx - 2);
      iy = min((int)fy, g.ny - 2);
      iz = min((int)fz, g.nz - 2);
      gc.ox = R(ix);
      gc.oy = R(iy);
      gc.oz = R(iz);
    }
    wx = fx - gc.ox;
    wy = fy - gc.oy;
    wz = fz - gc.oz;
    const size_t sx = 1, sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
    const size_t b = ((size_t)iz * g.ny + iy) * g.nx + ix;
    // raw corner values c[comp][corner], corner = cx + 2 cy + 4 cz
    if (g.packed) {
      // node-interleaved: two 16-byte loads per corner, one 32-byte sector
      const size_t off[8] = {b, b + sx, b + sy, b + sy + sx, b + sz, b + sz + sx, b + sz + sy,
                             b + sz + sy + sx};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 lo4 = __ldg(g.packed + 2 * off[k]);
        const float4 hi4 = __ldg(g.packed + 2 * off[k] + 1);
        gc.c[0][k] = lo4.x; gc.c[1][k] = lo4.y; gc.c[2][k] = lo4.z;
        gc.c[3][k] = lo4.w; gc.c[4][k] = hi4.x; gc.c[5][k] = hi4.y;
      }
    } else {
#pragma unroll
      for (int comp = 0; comp < 6; ++comp) {
        const float *f = g.f[comp] + b;
        R *c = gc.c[comp];
        c[0] = __ldg(f);
        c[1] = __ldg(f + sx);
        c[2] = __ldg(f + sy);
        c[3] = __ldg(f + sy + sx);
        c[4] = __ldg(f + sz);
        c[5] = __ldg(f + sz + sx);
        c[6] = __ldg(f + sz + sy);
        c[7] = __ldg(f + sz + sy + sx);
      }
    }
  }
  gc.wx = wx;
  gc.wy = wy;
  gc.wz = wz;
}

// The 8 trilinear weights of the cached cell, corner = cx + 2 cy + 4 cz.
template <typename R>
__device__ __forceinline__ void trilinear_weights(const GridCache<R> &gc, R w[8]) {
  const R wx = gc.wx, wy = gc.wy, wz = gc.wz;
  const R ux = R(1) - wx, uy = R(1) - wy, uz = R(1) - wz;
  const R a00 = ux * uy, a10 = wx * uy, a01 = ux * wy, a11 = wx * wy;
  w[0] = a00 * uz; w[1] = a10 * uz; w[2] = a01 * uz; w[3] = a11 * uz;
  w[4] = a00 * wz; w[5] = a10 * wz; w[6] = a01 * wz; w[7] = a11 * wz;
}

// Phase 2: add the interpolated grid field to E, B, straight from the raw
// corner values (no per-refetch conversion: a refetch by any lane would
// otherwise cost the whole warp the conversion).
template <typename R>
__device__ __forceinline__ void grid_eval(GridCache<R> &gc, R E[3], R B[3]) {
  R w[8];
  trilinear_weights(gc, w);
  R out[6];
#pragma unroll
  for (int comp = 0; comp < 6; ++comp) {
    const R *c = gc.c[comp];
    R r = w[0] * c[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) r = fma(w[k], c[k], r);
    out[comp] = r;
  }
  E[0] += out[0]; E[1] += out[1]; E[2] += out[2];
  B[0] += out[3]; B[1] += out[4]; B[2] += out[5];
}

// Both phases back to back.
template <typename R>
__device__ __forceinline__ void grid_gather(const GridView &g, GridCache<R> &gc, R x, R y, R z,
                                            R E[3], R B[3]) {
  grid_fetch(g, gc, x, y, z);
  grid_eval(gc, E, B);
}

// ---------------------------------------------- shared-memory cell cache
// The float kernels keep the current cell in shared memory instead of 48
// registers (which capped occupancy at ~18 warps per SM): 16 slots of 16
// bytes per thread, slot 2k = (Ex, Ey, Ez, Bx) and slot 2k+1 = (By, Bz, -, -)
// of corner k = cx + 2 cy + 4 cz, slots interleaved across the block so that
// a warp's 16-byte accesses are conflict-free.  A refetch is issued as
// asynchronous global->shared copies (cp.async, no register staging) at the
// start of the step and waited for just before the interpolation, after the
// analytic field, so the copy latency overlaps that work.
struct GridSlots {
  float ox, oy, oz;  // lower corner of the cached cell in grid units
  float wx, wy, wz;  // weights of the current step
  unsigned s0;       // shared-window address of this thread's slot 0
  unsigned step;     // bytes between consecutive slots of one thread
};

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ float4 lds128(unsigned addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

__device__ __forceinline__ void grid_slots_init(GridSlots &gc, void *slots_base) {
  gc.ox = gc.oy = gc.oz = -16.0f;
  gc.s0 = (unsigned)__cvta_generic_to_shared(slots_base) + 16u * threadIdx.x;
  gc.step = 16u * blockDim.x;
}

// Every lane of the warp calls this together (warp-uniform refetch branch).
__device__ __forceinline__ void grid_fetch(const GridView &g, GridSlots &gc, float x, float y,
                                           float z) {
  const float fx = grid_unit<float>(x, g.inv_d[0], g.off[0], g.top[0]);
  const float fy = grid_unit<float>(y, g.inv_d[1], g.off[1], g.top[1]);
  const float fz = grid_unit<float>(z, g.inv_d[2], g.off[2], g.top[2]);
  float wx = fx - gc.ox, wy = fy - gc.oy, wz = fz - gc.oz;
  // inside the cached cell (faces included) iff max |w - 1/2| <= 1/2
  const float dev = fmaxf(fabsf(wx - 0.5f), fmaxf(fabsf(wy - 0.5f), fabsf(wz - 0.5f)));
  const bool need = !(dev <= 0.5f);
  if (__any_sync(0xffffffffu, need) && need) {
    // lower cell corner without the conversion pipe (see the register cache)
    auto corner = [](float f, float top2, int &i) {
      float c = __fsub_rn(__fadd_rn(__fsub_rn(f, 0.5f), kRoundMagic), kRoundMagic);
      c = fminf(fmaxf(c, 0.0f), top2);
      i = __float_as_int(__fadd_rn(c, kRoundMagic)) - __float_as_int(kRoundMagic);
      return c;
    };
    int ix, iy, iz;
    gc.ox = corner(fx, g.top2[0], ix);
    gc.oy = corner(fy, g.top2[1], iy);
    gc.oz = corner(fz, g.top2[2], iz);
    wx = fx - gc.ox;
    wy = fy - gc.oy;
    wz = fz - gc.oz;
    const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
    const size_t b = ((size_t)iz * g.ny + iy) * g.nx + ix;
    const size_t off[8] = {b, b + 1, b + sy, b + sy + 1, b + sz, b + sz + 1, b + sz + sy,
                           b + sz + sy + 1};
    if (g.packed) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        cp_async16(gc.s0 + (2 * k) * gc.step, g.packed + 2 * off[k]);
        cp_async16(gc.s0 + (2 * k + 1) * gc.step, g.packed + 2 * off[k] + 1);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int comp = 0; comp < 6; ++comp)
          cp_async4(gc.s0 + (2 * k + comp / 4) * gc.step + 4u * (comp % 4), g.f[comp] + off[k]);
    }
  }
  gc.wx = wx;
  gc.wy = wy;
  gc.wz = wz;
}

__device__ __forceinline__ void grid_eval(const GridSlots &gc, float E[3], float B[3]) {
  cp_async_wait_all();  // this thread's copies (if any) have landed
  const float ux = 1.0f - gc.wx, uy = 1.0f - gc.wy, uz = 1.0f - gc.wz;
  const float a00 = ux * uy, a10 = gc.wx * uy, a01 = ux * gc.wy, a11 = gc.wx * gc.wy;
  const float w[8] = {a00 * uz, a10 * uz, a01 * uz, a11 * uz, a00 * gc.wz, a10 * gc.wz,
                      a01 * gc.wz, a11 * gc.wz};
  float o[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 lo = lds128(gc.s0 + (2 * k) * gc.step);
    const float4 hi = lds128(gc.s0 + (2 * k + 1) * gc.step);
    o[0] = fmaf(w[k], lo.x, o[0]);
    o[1] = fmaf(w[k], lo.y, o[1]);
    o[2] = fmaf(w[k], lo.z, o[2]);
    o[3] = fmaf(w[k], lo.w, o[3]);
    o[4] = fmaf(w[k], hi.x, o[4]);
    o[5] = fmaf(w[k], hi.y, o[5]);
  }
  E[0] += o[0]; E[1] += o[1]; E[2] += o[2];
  B[0] += o[3]; B[1] += o[4]; B[2] += o[5];
}

// ------------------------------------- shared-memory cell-coefficient cache
// With the per-cell coefficient copy (AP_PACK_CELLS) a thread keeps the 48
// coefficients of its current cell (12 float4, one 192-byte record) in
// registers or in 12 shared-memory slots, refetched as 12 contiguous 16-byte
// loads or cp.async copies.  The record interleaves the components in pairs
// (Ex, Ey), (Ez, Bx), (By, Bz): float4 4p + j holds coefficients 2j and
// 2j + 1 of both components of pair p, (a_2j, a'_2j, a_2j+1, a'_2j+1), so that
// each half of a float4 is a register pair and one packed FMA advances both
// components of a pair.  Per component (7 FMA)
//   F = a0 + a3 wz + wy (a2 + a5 wz) + wx (a1 + a6 wz + wy (a4 + a7 wz)),
// evaluated for the three pairs with 21 packed FMA; each half rounds as the
// scalar fmaf does, so the result per component is the scalar evaluation's.
__device__ __forceinline__ void cell_eval(const float4 c[12], float wx, float wy, float wz,
                                          float o[6]) {
  const float2 WX = make_float2(wx, wx), WY = make_float2(wy, wy), WZ = make_float2(wz, wz);
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const float4 q0 = c[4 * p], q1 = c[4 * p + 1], q2 = c[4 * p + 2], q3 = c[4 * p + 3];
    const float2 a0 = make_float2(q0.x, q0.y), a1 = make_float2(q0.z, q0.w);
    const float2 a2 = make_float2(q1.x, q1.y), a3 = make_float2(q1.z, q1.w);
    const float2 a4 = make_float2(q2.x, q2.y), a5 = make_float2(q2.z, q2.w);
    const float2 a6 = make_float2(q3.x, q3.y), a7 = make_float2(q3.z, q3.w);
    const float2 X = __ffma2_rn(a6, WZ, __ffma2_rn(__ffma2_rn(a7, WZ, a4), WY, a1));
    const float2 Y = __ffma2_rn(a5, WZ, a2);
    const float2 O = __ffma2_rn(X, WX, __ffma2_rn(Y, WY, __ffma2_rn(a3, WZ, a0)));
    o[2 * p] = O.x;
    o[2 * p + 1] = O.y;
  }
}

__device__ __forceinline__ size_t cell_index(const GridView &g, int ix, int iy, int iz) {
  return ((size_t)iz * (g.ny - 1) + iy) * (g.nx - 1) + ix;
}

// The cell of a particle at grid units (fx, fy, fz) for a refetch: its lower
// corner (o), the weights inside it (w) and its index.  The corner comes
// without the conversion pipe: rint(f - 1/2) through the 1.5 * 2^23 magic
// number (a face point may land in the cell below, where its weight is 1:
// same value), clamped to [0, n - 2]; the integer is read from the bits of
// (corner + magic).
__device__ __forceinline__ size_t locate_cell(const GridView &g, float fx, float fy, float fz,
                                              float &ox, float &oy, float &oz, float &wx, float &wy,
                                              float &wz) {
  auto corner = [](float f, float top2, int &i) {
    float c = __fsub_rn(__fadd_rn(__fsub_rn(f, 0.5f), kRoundMagic), kRoundMagic);
    c = fminf(fmaxf(c, 0.0f), top2);
    i = __float_as_int(__fadd_rn(c, kRoundMagic)) - __float_as_int(kRoundMagic);
    return c;
  };
  int ix, iy, iz;
  ox = corner(fx, g.top2[0], ix);
  oy = corner(fy, g.top2[1], iy);
  oz = corner(fz, g.top2[2], iz);
  wx = fx - ox;
  wy = fy - oy;
  wz = fz - oz;
  return cell_index(g, ix, iy, iz);
}

// Slot k of thread t lies at 16 t + k kCellSlotStride: a compile-time stride
// (room for blocks of up to 256 threads), so the 12 slot addresses of a step
// are immediate offsets from one register.
constexpr unsigned kCellSlotStride = 16u * 256u;

struct CellSlots {
  float ox, oy, oz;  // lower corner of the cached cell in grid units
  float wx, wy, wz;  // weights of the current step
  unsigned s0;       // shared-window address of this thread's slot 0
};

__device__ __forceinline__ void grid_slots_init(CellSlots &gc, void *slots_base) {
  gc.ox = gc.oy = gc.oz = -16.0f;
  gc.s0 = (unsigned)__cvta_generic_to_shared(slots_base) + 16u * threadIdx.x;
}

// The record of the cell at grid units (fx, fy, fz) into the cache, and the
// weights inside it: 12 16-byte cp.async copies into the thread's slots.
__device__ __forceinline__ void cell_refetch(const GridView &g, CellSlots &gc, float fx, float fy, float fz,
                                             float &wx, float &wy, float &wz) {
  const size_t cell = locate_cell(g, fx, fy, fz, gc.ox, gc.oy, gc.oz, wx, wy, wz);
  const float4 *src = g.cells + 12 * cell;
#pragma unroll
  for (int k = 0; k < 12; ++k) cp_async16(gc.s0 + k * kCellSlotStride, src + k);
}

// Every lane of the warp calls this together (warp-uniform refetch branch).
__device__ __forceinline__ void grid_fetch(const GridView &g, CellSlots &gc, float x, float y,
                                           float z) {
  const float fx = grid_unit<float>(x, g.inv_d[0], g.off[0], g.top[0]);
  const float fy = grid_unit<float>(y, g.inv_d[1], g.off[1], g.top[1]);
  const float fz = grid_unit<float>(z, g.inv_d[2], g.off[2], g.top[2]);
  float wx = fx - gc.ox, wy = fy - gc.oy, wz = fz - gc.oz;
  // inside the cached cell (faces included) iff max |w - 1/2| <= 1/2
  const float dev = fmaxf(fabsf(wx - 0.5f), fmaxf(fabsf(wy - 0.5f), fabsf(wz - 0.5f)));
  const bool need = !(dev <= 0.5f);
  if (__any_sync(0xffffffffu, need) && need) cell_refetch(g, gc, fx, fy, fz, wx, wy, wz);
  gc.wx = wx;
  gc.wy = wy;
  gc.wz = wz;
}

// the six interpolated components from the cached cell (the caller has
// waited for the cell's copies)
__device__ __forceinline__ void grid_values(const CellSlots &gc, float o[6]) {
  float4 c[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) c[k] = lds128(gc.s0 + k * kCellSlotStride);
  cell_eval(c, gc.wx, gc.wy, gc.wz, o);
}

__device__ __forceinline__ void grid_eval(const CellSlots &gc, float E[3], float B[3]) {
  cp_async_wait_all();  // this thread's copies (if any) have landed
  float o[6];
  grid_values(gc, o);
  E[0] += o[0]; E[1] += o[1]; E[2] += o[2];
  B[0] += o[3]; B[1] += o[4]; B[2] += o[5];
}

// The same coefficients held in 48 registers instead (grid_cache = 1): a
// refetch is 12 16-byte loads into the cache registers, issued at the start
// of the step and consumed after the analytic field; no shared memory.
struct CellRegs {
  float ox, oy, oz;
  float wx, wy, wz;
  float4 c[12];
};

__device__ __forceinline__ void grid_slots_init(CellRegs &gc, void *) {
  gc.ox = gc.oy = gc.oz = -16.0f;
#pragma unroll
  for (int k = 0; k < 12; ++k) gc.c[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// The same into the cache registers: 12 16-byte loads.
__device__ __forceinline__ void cell_refetch(const GridView &g, CellRegs &gc, float fx, float fy, float fz,
                                             float &wx, float &wy, float &wz) {
  const size_t cell = locate_cell(g, fx, fy, fz, gc.ox, gc.oy, gc.oz, wx, wy, wz);
  const float4 *src = g.cells + 12 * cell;
#pragma unroll
  for (int k = 0; k < 12; ++k) gc.c[k] = __ldg(src + k);
}

__device__ __forceinline__ void grid_fetch(const GridView &g, CellRegs &gc, float x, float y,
                                           float z) {
  const float fx = grid_unit<float>(x, g.inv_d[0], g.off[0], g.top[0]);
  const float fy = grid_unit<float>(y, g.inv_d[1], g.off[1], g.top[1]);
  const float fz = grid_unit<float>(z, g.inv_d[2], g.off[2], g.top[2]);
  float wx = fx - gc.ox, wy = fy - gc.oy, wz = fz - gc.oz;
  // inside the cached cell (faces included) iff max |w - 1/2| <= 1/2
  const float dev = fmaxf(fabsf(wx - 0.5f), fmaxf(fabsf(wy - 0.5f), fabsf(wz - 0.5f)));
  const bool need = !(dev <= 0.5f);
  if (__any_sync(0xffffffffu, need) && need) cell_refetch(g, gc, fx, fy, fz, wx, wy, wz);
  gc.wx = wx;
  gc.wy = wy;
  gc.wz = wz;
}

__device__ __forceinline__ void grid_values(const CellRegs &gc, float o[6]) {
  cell_eval(gc.c, gc.wx, gc.wy, gc.wz, o);
}

__device__ __forceinline__ void grid_eval(const CellRegs &gc, float E[3], float B[3]) {
  float o[6];
  grid_values(gc, o);
  E[0] += o[0]; E[1] += o[1]; E[2] += o[2];
  B[0] += o[3]; B[1] += o[4]; B[2] += o[5];
}

// ------------------------------------------------------------ Boris push
// Relativistic Boris step (Boris 1970) for charge -1, mass 1: half electric
// kick, rotation about B with tan(angle/2) = |tau|, half electric kick.
// Returns 1/gamma of the new momentum.
template <typename R>
__device__ __forceinline__ R boris(R u[3], const R E[3], const R B[3], R dt) {
  const R h = R(-0.5) * dt;
  R um0 = fma(h, E[0], u[0]), um1 = fma(h, E[1], u[1]), um2 = fma(h, E[2], u[2]);
  R ig = rsqrt_r(fma(um0, um0, fma(um1, um1, fma(um2, um2, R(1)))));
  R hg = h * ig;
  R t0 = hg * B[0], t1 = hg * B[1], t2 = hg * B[2];
  R tt = fma(t0, t0, fma(t1, t1, t2 * t2));
  R sc = R(2) * rcp_r(R(1) + tt);
  R s0 = sc * t0, s1 = sc * t1, s2 = sc * t2;
  R p0 = um0 + (um1 * t2 - um2 * t1);
  R p1 = um1 + (um2 * t0 - um0 * t2);
  R p2 = um2 + (um0 * t1 - um1 * t0);
  R q0 = um0 + (p1 * s2 - p2 * s1);
  R q1 = um1 + (p2 * s0 - p0 * s2);
  R q2 = um2 + (p0 * s1 - p1 * s0);
  u[0] = fma(h, E[0], q0);
  u[1] = fma(h, E[1], q1);
  u[2] = fma(h, E[2], q2);
  return rsqrt_r(fma(u[0], u[0], fma(u[1], u[1], fma(u[2], u[2], R(1)))));
}

__device__ __forceinline__ bool all_finite(double a, double b, double c, double d, double e,
                                           double f) {
  return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d) && isfinite(e) && isfinite(f);
}

// warp max of a non-negative float, one atomic per warp into a double slot
__device__ __forceinline__ void warp_max_to(double *slot, float v, unsigned mask) {
  unsigned bits = __float_as_uint(v);
  bits = __reduce_max_sync(mask, bits);
  if ((threadIdx.x & 31) == (__ffs(mask) - 1)) {
    double d = (double)__uint_as_float(bits);
    atomicMax(reinterpret_cast<unsigned long long *>(slot),
              (unsigned long long)__double_as_longlong(d));
  }
}
__device__ __forceinline__ void warp_max_to(double *slot, double v, unsigned mask) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(mask, bits, o);
    // lanes outside the mask return their own value; max is unaffected
    if (other > bits) bits = other;
  }
  if ((threadIdx.x & 31) == (__ffs(mask) - 1))
    atomicMax(reinterpret_cast<unsigned long long *>(slot), bits);
}

}  // namespace apt
