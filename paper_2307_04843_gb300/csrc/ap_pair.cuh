// ap_pair.cuh -- arithmetic on pairs of floats, for push kernels in which one
// thread carries two particles through the step loop.
//
// The sm_100 family has packed FP32 instructions (add, mul and fma on .f32x2
// register pairs): one instruction performs the same operation for both
// halves.  The FP32 pipe's lane throughput is the same as with scalar
// instructions (on GB300 both reach ~120 lane operations per clock per SM),
// so what a packed instruction saves is an issue slot -- and instruction
// issue, not the FP32 pipe, is what bounds the one-particle push kernels.
// With the two particles of a thread in the two halves of every value, all
// the FP32 arithmetic of the field evaluation, the Boris step and the
// position update pairs up without any shuffling; the special-function (MUFU)
// operations stay one per particle.
//
// Every packed operation rounds each half exactly as the scalar _rn
// intrinsic does (round to nearest even, no contraction), so the error-free
// transformations of the float-float phase and position carry over
// unchanged.
#pragma once

#include "ap_device.cuh"

namespace apt {

// The pair type and its operations live in a namespace of their own: they
// are found by argument-dependent lookup for pair arguments only, so they
// never hide the scalar fma, fabs, ... that the rest of the library calls.
namespace pair {

struct __align__(8) F2 {
  float x, y;
  F2() = default;
  // a scalar broadcast to both halves (pulse constants, literals)
  __device__ __forceinline__ F2(float s) : x(s), y(s) {}
  __device__ __forceinline__ F2(float a, float b) : x(a), y(b) {}
};

__device__ __forceinline__ float2 f2v(F2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ F2 f2of(float2 v) { return F2(v.x, v.y); }

// Negating a pair is not free (no packed negate; the compiler emits extra
// instructions for about two thirds of them), so the code below subtracts
// with the packed sub and negates constants rather than variables.
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2of(__fadd2_rn(f2v(a), f2v(b))); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.x, -a.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return f2of(__fmul2_rn(f2v(a), f2v(b))); }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
  return f2of(__ffma2_rn(f2v(a), f2v(b), f2v(c)));
}
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2 &operator*=(F2 &a, F2 b) { return a = a * b; }
// true when either half differs (used only where both halves may then take
// the same path: a factor that is exactly 1 for the other half)
__device__ __forceinline__ bool operator!=(F2 a, F2 b) { return a.x != b.x || a.y != b.y; }
__device__ __forceinline__ F2 fabs(F2 a) { return F2(fabsf(a.x), fabsf(a.y)); }

// the spelling of the fused operation that the float-float code uses
__device__ __forceinline__ F2 fma_rn(F2 a, F2 b, F2 c) { return fma(a, b, c); }

// special-function unit: one MUFU operation per half
__device__ __forceinline__ F2 rcp_r(F2 a) { return F2(mufu_rcp(a.x), mufu_rcp(a.y)); }
__device__ __forceinline__ F2 rsqrt_r(F2 a) { return F2(mufu_rsqrt(a.x), mufu_rsqrt(a.y)); }
__device__ __forceinline__ F2 exp2_r(F2 a) { return F2(mufu_ex2(a.x), mufu_ex2(a.y)); }
__device__ __forceinline__ F2 cos_r(F2 a) { return F2(mufu_cos(a.x), mufu_cos(a.y)); }
__device__ __forceinline__ void sincos_r(F2 a, F2 *s, F2 *c) {
  *s = F2(mufu_sin(a.x), mufu_sin(a.y));
  *c = F2(mufu_cos(a.x), mufu_cos(a.y));
}

__device__ __forceinline__ Cx<F2> cscale(Cx<F2> a, F2 s) { return {a.re * s, a.im * s}; }

// sin^2 envelope value m, cleared in each half whose |eta| lies beyond the
// window's half-width b
__device__ __forceinline__ F2 sin2_window(F2 m, F2 eta, float b) {
  return F2(fabsf(eta.x) > b ? 0.0f : m.x, fabsf(eta.y) > b ? 0.0f : m.y);
}

// complex product with two fused operations per part
__device__ __forceinline__ Cx<F2> cmul(Cx<F2> a, Cx<F2> b) {
  return {fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re)};
}

// round to the nearest integer through the 1.5 * 2^23 magic number, valid for
// |a b| < 2^22 (see round_fma)
__device__ __forceinline__ F2 round_fma(F2 a, F2 b) {
  return fma(a, b, F2(kRoundMagic)) - F2(kRoundMagic);
}

// argument reduction of a moderate angle (a few times 2 pi), as reduce_f
__device__ __forceinline__ F2 reduce_f(F2 x) {
  const F2 m = round_fma(x, F2(kInvTwoPi));
  x = fma(m, F2(-kTwoPiHi), x);
  return fma(m, F2(-kTwoPiLo), x);
}

// ------------------------------------------------------------ float-float
struct FF2 {
  F2 hi, lo;
};

__device__ __forceinline__ FF2 two_sum(F2 a, F2 b) {
  const F2 s = a + b;
  const F2 bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

// a - b as hi + lo (the TwoSum of a and -b)
__device__ __forceinline__ FF2 two_diff(F2 a, F2 b) {
  const F2 s = a - b;
  const F2 bb = s - a;
  return {s, (a - (s - bb)) - (b + bb)};
}

__device__ __forceinline__ FF2 two_prod(F2 a, F2 b) {
  const F2 p = a * b;
  return {p, fma(a, b, -p)};
}

// The product a b = p + e with the error's sign flipped, from the negated
// constant factor nb = -b: n = fma(a, nb, p) = p - a b exactly = -e.
__device__ __forceinline__ F2 two_prod_nerr(F2 a, F2 nb, F2 p) { return fma(a, nb, p); }

// (hi + lo) reduced modulo 2 pi (Cody-Waite, two constants), as reduce_ff:
// r = hi - m P1 exactly (m P1 = p + e), t = (lo - e) - m P2
__device__ __forceinline__ F2 reduce_ff(F2 hi, F2 lo) {
  const F2 m = round_fma(hi, F2(kInvTwoPi));
  const F2 p = m * F2(kTwoPiHi);
  const F2 ne = two_prod_nerr(m, F2(-kTwoPiHi), p);
  const F2 r = hi - p;
  const F2 t = fma(m, F2(-kTwoPiLo), lo + ne);
  return r + t;
}

}  // namespace pair

using pair::F2;
using pair::FF2;

template <>
struct IsPair<F2> : std::true_type {};

// Positions of the two particles of a thread as float-float pairs, the same
// compensated accumulation as Pos<AP_FP32_PHASEFF>.  The longitudinal
// coordinate is held relative to the pulse's focus, dz = z - z_f (formed in
// double on load), since the carrier phase needs dz to float-float accuracy
// every step and the absolute z only in float (for the grid).
struct Pos2 {
  FF2 x, y, dz;
  __device__ __forceinline__ void load(const double X[2], const double Y[2], const double Z[2], double zf) {
    const FF a = split_double(X[0]), b = split_double(X[1]);
    x = {F2(a.hi, b.hi), F2(a.lo, b.lo)};
    const FF c = split_double(Y[0]), d = split_double(Y[1]);
    y = {F2(c.hi, d.hi), F2(c.lo, d.lo)};
    const FF e = split_double(Z[0] - zf), f = split_double(Z[1] - zf);
    dz = {F2(e.hi, f.hi), F2(e.lo, f.lo)};
  }
  __device__ __forceinline__ static void acc(FF2 &p, F2 d) {
    const F2 y = d + p.lo;
    const F2 t = p.hi + y;
    p.lo = y - (t - p.hi);
    p.hi = t;
  }
  __device__ __forceinline__ void advance(F2 vx, F2 vy, F2 vz, F2 dt_xy, F2 dt) {
    acc(x, dt_xy * vx);
    acc(y, dt_xy * vy);
    acc(dz, dt * vz);
  }
  __device__ __forceinline__ F2 xr() const { return x.hi + x.lo; }
  __device__ __forceinline__ F2 yr() const { return y.hi + y.lo; }
  // absolute z in float, from z_f = zf_hi + zf_lo
  __device__ __forceinline__ F2 zr(float zf_hi, float zf_lo) const {
    return (dz.hi + F2(zf_hi)) + (dz.lo + F2(zf_lo));
  }
};

// Local coordinates of both particles at one step (float-float phase), the
// pairwise form of local_coords<AP_FP32_PHASEFF>: the step's time base `st`
// is shared by the two particles.
__device__ __forceinline__ Local<F2> local_coords2(const Pulse<float> &P, const StepFF &st,
                                                   const Pos2 &pos) {
  Local<F2> L;
  const FF2 dz = pos.dz;  // z - z_f
  // psi = C_n - k dz, k dz = kp + ke with -ke from the negated constant
  const F2 kp = F2(P.k_hi) * dz.hi;
  const F2 nke = two_prod_nerr(dz.hi, F2(-P.k_hi), kp);
  const F2 kdlo = fma(F2(P.k_hi), dz.lo, F2(P.k_lo) * dz.hi) - nke;
  const FF2 ps = two_diff(F2(st.C), kp);
  L.psi = reduce_ff(ps.hi, ps.lo - kdlo);
  L.x = pos.xr();
  L.y = pos.yr();
  L.dz = dz.hi + dz.lo;
  const float Tf = __fadd_rn(st.Th, st.Tl);
  L.eta = fma(L.dz, F2(-P.inv_vg), F2(Tf));
  L.T = F2(Tf);
  // phi' = T - dz as float-float
  const FF2 ph = two_diff(F2(st.Th), dz.hi);
  L.phi_hi = ph.hi;
  L.phi_lo = ph.lo + (F2(st.Tl) - dz.lo);
  return L;
}

// The cell test and weights of a thread's two particles with packed
// arithmetic (grid units, offsets from each cached cell), then each
// particle's own warp-uniform refetch branch, as grid_fetch does per particle.
// gk: the grid's inverse spacings and offsets pre-broadcast in shared memory,
// gk[a] = (inv_d[a], inv_d[a], off[a], off[a]), and gk[3] = (1/2, 1/2, -, -):
// a 16-byte load yields both pair operands, where constants kept in the
// kernel parameters would be re-broadcast into register pairs every step
// (the two-particle kernels run at their register limit).
template <class CA, class CB>
__device__ __forceinline__ void grid_fetch2(const GridView &g, CA &ga, CB &gb, F2 x, F2 y, F2 z,
                                            const float4 *gk) {
  const float4 kx = gk[0], ky = gk[1], kz = gk[2], kh = gk[3];
  F2 f[3] = {fma(x, F2(kx.x, kx.y), F2(kx.z, kx.w)), fma(y, F2(ky.x, ky.y), F2(ky.z, ky.w)),
             fma(z, F2(kz.x, kz.y), F2(kz.z, kz.w))};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    f[a] = F2(fminf(fmaxf(f[a].x, 0.0f), g.top[a]), fminf(fmaxf(f[a].y, 0.0f), g.top[a]));
  F2 w[3] = {f[0] - F2(ga.ox, gb.ox), f[1] - F2(ga.oy, gb.oy), f[2] - F2(ga.oz, gb.oz)};
  // inside the cached cell (faces included) iff max |w - 1/2| <= 1/2
  const F2 half(kh.x, kh.y);
  const F2 d0 = w[0] - half, d1 = w[1] - half, d2 = w[2] - half;
  const bool need_a = !(fmaxf(fabsf(d0.x), fmaxf(fabsf(d1.x), fabsf(d2.x))) <= 0.5f);
  const bool need_b = !(fmaxf(fabsf(d0.y), fmaxf(fabsf(d1.y), fabsf(d2.y))) <= 0.5f);
  float wa[3] = {w[0].x, w[1].x, w[2].x}, wb[3] = {w[0].y, w[1].y, w[2].y};
  if (__any_sync(0xffffffffu, need_a) && need_a) cell_refetch(g, ga, f[0].x, f[1].x, f[2].x, wa[0], wa[1], wa[2]);
  if (__any_sync(0xffffffffu, need_b) && need_b) cell_refetch(g, gb, f[0].y, f[1].y, f[2].y, wb[0], wb[1], wb[2]);
  ga.wx = wa[0]; ga.wy = wa[1]; ga.wz = wa[2];
  gb.wx = wb[0]; gb.wy = wb[1]; gb.wz = wb[2];
}

}  // namespace apt
