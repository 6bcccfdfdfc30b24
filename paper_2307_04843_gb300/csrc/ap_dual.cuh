// ap_dual.cuh -- forward-mode dual numbers for the field Jacobian of the
// adjoint (row a13).
//
// Dual<R, N> carries a value and N tangents.  The field functions of
// ap_device.cuh are templated on the scalar type, so instantiating them with
// Dual<float, 4> seeded in (x, y, z - z_f, w0) -- Dual<float, 5> with beta_f
// added for the closed-form flying focus -- yields the fields and their
// derivatives with respect to the particle position, the focal position
// (d/dz_f = -d/d(z - z_f)), the waist and the focal velocity in one pass,
// with exactly the arithmetic of the forward push for the value part.
#pragma once

#include <type_traits>

#include "ap_device.cuh"

namespace apt {

// keep the plain-number overloads visible next to the dual ones below
using ::fabs;
using ::fma;

template <typename R, int N>
struct Dual {
  R v;
  R d[N];
  __device__ __forceinline__ Dual() {}
  template <typename T, typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
  __device__ __forceinline__ Dual(T x) : v(R(x)) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = R(0);
  }
  __device__ __forceinline__ static Dual seed(R x, int k, R dk = R(1)) {
    Dual r(x);
    r.d[k] = dk;
    return r;
  }
  __device__ __forceinline__ Dual &operator*=(const Dual &b) { return *this = *this * b; }
  __device__ __forceinline__ Dual &operator+=(const Dual &b) { return *this = *this + b; }
};

template <class T>
struct is_dual : std::false_type {};
template <typename R, int N>
struct is_dual<Dual<R, N>> : std::true_type {};

template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator+(const Dual<R, N> &a, const Dual<R, N> &b) {
  Dual<R, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N> &a, const Dual<R, N> &b) {
  Dual<R, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N> &a) {
  Dual<R, N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> operator*(const Dual<R, N> &a, const Dual<R, N> &b) {
  Dual<R, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
// mixed with a plain number (promoted to a constant dual)
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ Dual<R, N> operator*(const Dual<R, N> &a, T b) {
  Dual<R, N> r;
  r.v = a.v * R(b);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * R(b);
  return r;
}
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ Dual<R, N> operator*(T b, const Dual<R, N> &a) {
  return a * b;
}
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ Dual<R, N> operator+(const Dual<R, N> &a, T b) {
  Dual<R, N> r = a;
  r.v = a.v + R(b);
  return r;
}
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ Dual<R, N> operator+(T b, const Dual<R, N> &a) {
  return a + b;
}
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N> &a, T b) {
  Dual<R, N> r = a;
  r.v = a.v - R(b);
  return r;
}
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ Dual<R, N> operator-(T b, const Dual<R, N> &a) {
  return -(a - b);
}
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ bool operator>(const Dual<R, N> &a, T b) {
  return a.v > R(b);
}
template <typename R, int N, typename T,
          typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ bool operator!=(const Dual<R, N> &a, T b) {
  return a.v != R(b);
}
template <typename R, int N>
__device__ __forceinline__ bool operator!=(const Dual<R, N> &a, const Dual<R, N> &b) {
  return a.v != b.v;
}

// fma with any mix of dual and plain arguments
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> fma_d(const Dual<R, N> &a, const Dual<R, N> &b,
                                            const Dual<R, N> &c) {
  Dual<R, N> r;
  r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fma(a.d[i], b.v, fma(a.v, b.d[i], c.d[i]));
  return r;
}
template <typename A, typename B, typename C,
          typename = typename std::enable_if<is_dual<A>::value || is_dual<B>::value ||
                                             is_dual<C>::value>::type>
__device__ __forceinline__ auto fma(const A &a, const B &b, const C &c) {
  using D = typename std::conditional<is_dual<A>::value, A,
                                      typename std::conditional<is_dual<B>::value, B, C>::type>::type;
  return fma_d(D(a), D(b), D(c));
}

template <typename R, int N>
__device__ __forceinline__ Dual<R, N> fabs(const Dual<R, N> &a) {
  return a.v < R(0) ? -a : a;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> rcp_r(const Dual<R, N> &a) {
  Dual<R, N> r;
  r.v = rcp_r(a.v);
  const R s = -r.v * r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> exp2_r(const Dual<R, N> &a) {
  Dual<R, N> r;
  r.v = exp2_r(a.v);
  const R s = r.v * R(0.69314718055994531);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}
template <typename R, int N>
__device__ __forceinline__ void sincos_r(const Dual<R, N> &a, Dual<R, N> *s, Dual<R, N> *c) {
  R sv, cv;
  sincos_r(a.v, &sv, &cv);
  s->v = sv;
  c->v = cv;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    s->d[i] = cv * a.d[i];
    c->d[i] = -sv * a.d[i];
  }
}
template <typename R, int N>
__device__ __forceinline__ Dual<R, N> cos_r(const Dual<R, N> &a) {
  Dual<R, N> s, c;
  sincos_r(a, &s, &c);
  return c;
}

// reduction by whole turns changes no derivative
template <>
__device__ __forceinline__ Dual<float, 4> reduce_angle<Dual<float, 4>>(Dual<float, 4> a) {
  a.v = reduce_f(a.v);
  return a;
}
template <>
__device__ __forceinline__ Dual<float, 5> reduce_angle<Dual<float, 5>>(Dual<float, 5> a) {
  a.v = reduce_f(a.v);
  return a;
}

}  // namespace apt
