// ap_line.cu -- 1-D lines with a linear cold-plasma current (Sec. 4, the
// analytic pulse technique with an analytic current J1).
//
// Two updates of one line carrying E_x on the whole nodes z_k, B_y on the
// half nodes and the current J_x on the whole nodes at half time levels:
//   traditional: the Yee scheme of Sec. 2.1 with the current advanced by the
//     leapfrog dJ/dt = omega_p^2 E (the simulation Sec. 4 compares with);
//   split (APT): E, B hold the internally advanced E2, B2; the physical
//     current J is driven by E1 + E2, and E2 is sourced by J - J1, with the
//     analytic E1 (at t_n) and J1 (at t_n + dt/2) of a plane-wave pulse
//     evaluated in the kernel every step (Eqs. E_1_j, E_2_j, j1).
//
// One block per line; the line (E, B, J and a_k = dt omega_p^2(z_k)) stays
// on chip for all n_steps and is written back once: in registers for the
// traditional float line up to 6144 nodes (plasma_line_reg_kernel), in
// shared memory otherwise (line_kernel).  Per step of line_kernel: the
// B half step; a barrier; the current and E update of each node (one pass:
// both read only the node's own E and J and the neighbouring B); a barrier;
// the second B half step.  The second B half step and the next step's first
// one write only their own node and read only E, so no barrier separates
// them.  Each product, sum and difference is rounded separately in the
// stated order, so the double traditional line reproduces a plain double
// loop of the same expressions bit for bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "ap_kernels.cuh"

namespace apt {
namespace {

constexpr int kLineBlock = 1024;

__device__ __forceinline__ double l_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double l_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double l_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float l_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float l_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float l_mul(float a, float b) { return __fmul_rn(a, b); }

// Float-float split line: the node-dependent part of the carrier phase,
// k (z_k - z_f) as float-float, and z_k - z_f, computed once per launch with
// the operations of local_coords (so the phase and envelope argument of every
// evaluation are those of the generic path bit for bit).
struct NodeFF {
  float kd_hi, kd_lo, dz;
};

__device__ __forceinline__ NodeFF node_ff(const Pulse<float> &P, const LineArgs &a, float fk) {
  const FF z = node_coord_ff(fk, a.z0_hi, a.z0_lo, a.dz_hi, a.dz_lo);
  FF dz = two_sum(z.hi, -P.zf_hi);
  dz.lo = __fadd_rn(dz.lo, __fsub_rn(z.lo, P.zf_lo));
  FF kd = two_prod(P.k_hi, dz.hi);
  kd.lo = __fadd_rn(kd.lo, __fmaf_rn(P.k_hi, dz.lo, __fmul_rn(P.k_lo, dz.hi)));
  return {kd.hi, kd.lo, __fadd_rn(dz.hi, dz.lo)};
}

// E1 at t_n and J1 at t_n + dt/2 at two nodes of the float split line at once
// (the halves of every packed value, ap_pair.cuh: one issue slot per FP32
// operation for both nodes, the MUFU operations one per node), for a plane
// wave polarised along x (Eqs. plane_func, j1): the J1 carrier phase is the
// E1 phase advanced by omega dt/2, applied as a fixed rotation (sin, cos of
// omega dt/2 in sdl, cdl); the envelope and its log-derivatives are evaluated
// at eta and eta + dt/2.
__device__ __forceinline__ void line_sources_ff2(const Pulse<float> &P, const StepFF &st, F2 kd_hi, F2 kd_lo,
                                                 F2 dz, float sdl, float cdl, float hdt, F2 &E1, F2 &J1) {
  const FF2 ps = two_diff(F2(st.C), kd_hi);
  const F2 psi = reduce_ff(ps.hi, ps.lo - kd_lo);
  const float Tf = __fadd_rn(st.Th, st.Tl);
  const F2 eta0 = fma(dz, F2(-P.inv_vg), F2(Tf));
  F2 mul, l2;
  envelope(P, eta0, mul, l2);
  F2 a = F2(P.amp) * mul;
  if (l2 != F2(0.0f)) a *= exp2_r(l2);  // exp2(0) = 1 exactly for a half without an exponent
  F2 s, c;
  sincos_r(psi, &s, &c);
  E1 = a * c;
  const F2 eta = eta0 + F2(hdt);
  envelope(P, eta, mul, l2);
  F2 aj = F2(P.jamp * P.amp) * mul;
  if (l2 != F2(0.0f)) aj *= exp2_r(l2);
  const F2 sj = fma(s, F2(cdl), c * F2(sdl)), cj = fma(s, F2(-sdl), c * F2(cdl));
  F2 L1, L2;
  envelope_logd(P, eta, L1, L2);
  const Cx<F2> V = finite_duration(Cx<F2>{aj * cj, aj * sj}, 1.0f, L1, L2, P.inv_w);
  J1 = V.im;  // Re[p (-i V)] with p = (1, 0)
}

// Local coordinates of node k (x = y = 0) at one time level (double).
template <int PREC>
__device__ __forceinline__ Local<Real<PREC>> node_local(const Pulse<Real<PREC>> &P, const LineArgs &a,
                                                        const typename TimeBase<PREC>::Step &st, int k) {
  Pos<PREC> pos;
  if constexpr (PREC == AP_FP32_PHASEFF) {
    pos.x = FF{0.0f, 0.0f};
    pos.y = FF{0.0f, 0.0f};
    pos.z = node_coord_ff((float)k, a.z0_hi, a.z0_lo, a.dz_hi, a.dz_lo);
  } else {
    pos.load(0.0, 0.0, __dadd_rn(a.z0, __dmul_rn((double)k, a.dz)));
  }
  return local_coords<PREC>(P, st, pos);
}

template <typename T, int PREC, bool APT>
__global__ void __launch_bounds__(kLineBlock) line_kernel(const __grid_constant__ Pulse<Real<PREC>> P,
                                                          const __grid_constant__ LineArgs a) {
  using R = Real<PREC>;
  extern __shared__ __align__(16) unsigned char line_smem[];
  const int nz = a.nz;
  T *e = reinterpret_cast<T *>(line_smem);
  T *b = e + nz;
  T *j = b + nz;
  T *q = j + nz;  // a_k = dt omega_p^2(z_k)
  // float split line only: per-node phase constants (see NodeFF)
  constexpr bool kFF = APT && PREC == AP_FP32_PHASEFF;
  float *kdh = reinterpret_cast<float *>(q + nz);
  float *kdl = kdh + nz;
  float *dzn = kdl + nz;
  const size_t off = (size_t)blockIdx.x * (size_t)nz;
  T *Eg = static_cast<T *>(a.E) + off;
  T *Bg = static_cast<T *>(a.B) + off;
  T *Jg = static_cast<T *>(a.J) + off;
  const T *W = a.wp2 ? static_cast<const T *>(a.wp2) + off : nullptr;
  const T dt = (T)a.dt;
  const T r = (T)(a.dt / a.dz);
  const T hr = (T)(0.5 * (a.dt / a.dz));
  const T wpu = (T)a.omega_p2;
  const int t = threadIdx.x, bd = blockDim.x;
  for (int k = t; k < nz; k += bd) {
    e[k] = Eg[k];
    b[k] = Bg[k];
    j[k] = Jg[k];
    q[k] = l_mul(dt, W ? W[k] : wpu);
    if constexpr (kFF) {
      const NodeFF c = node_ff(P, a, (float)k);
      kdh[k] = c.kd_hi;
      kdl[k] = c.kd_lo;
      dzn[k] = c.dz;
    }
  }
  TimeBase<PREC> tb;
  if constexpr (APT) tb.init(P, a.t0, 0.5 * a.dt);  // level 2n: t_n, 2n + 1: t_n + dt/2
  float lev = 0.0f;  // 2n in float (exact: 2 n_steps + 1 < 2^24 is checked on the host)
  float sdl = 0.0f, cdl = 1.0f;  // sin, cos of omega dt/2 (float split line)
  if constexpr (kFF) {
    double sd, cd;
    sincos(0.5 * P.omega * a.dt, &sd, &cd);
    sdl = (float)sd;
    cdl = (float)cd;
  }
  const float hdt = (float)(0.5 * a.dt);
  __syncthreads();
  for (long long n = 0; n < a.n_steps; ++n) {
    // B^{n+1/2} = B^n - (r/2)(E_{k+1}^n - E_k^n)
    for (int k = t; k < nz - 1; k += bd) b[k] = l_sub(b[k], l_mul(hr, l_sub(e[k + 1], e[k])));
    __syncthreads();
    typename TimeBase<PREC>::Step st_e{}, st_j{};
    if constexpr (kFF) {
      st_e = tb.at_f(lev);
      lev += 2.0f;
    } else if constexpr (APT) {
      st_e = tb.at(2 * n);
      st_j = tb.at(2 * n + 1);
    }
    // J^{n+1/2} = J^{n-1/2} + a_k (E1 + E2)^n;  E^{n+1} = (E^n - r dB) - dt (J - J1)^{n+1/2}
    if constexpr (kFF) {
      // the thread's nodes k and k + bd in the two halves of one packed
      // source evaluation; each node's update as below
      auto update = [&](int k, float e1, float j1) {
        const T ek = e[k];
        const T jk = l_add(j[k], l_mul(q[k], l_add(e1, ek)));
        j[k] = jk;
        if (k >= 1) e[k] = l_sub(l_sub(ek, l_mul(r, l_sub(b[k], b[k - 1]))), l_mul(dt, l_sub(jk, j1)));
      };
      for (int k = t; k < nz; k += 2 * bd) {
        const int k2 = k + bd;
        const bool two = k2 < nz;
        const int kk = two ? k2 : k;  // the second half repeats node k when k + bd is past the line
        F2 e1, j1;
        line_sources_ff2(P, st_e, F2(kdh[k], kdh[kk]), F2(kdl[k], kdl[kk]), F2(dzn[k], dzn[kk]), sdl, cdl, hdt,
                         e1, j1);
        update(k, e1.x, j1.x);
        if (two) update(k2, e1.y, j1.y);
      }
    } else
    for (int k = t; k < nz; k += bd) {
      const T ek = e[k];
      T drive = ek;
      if constexpr (APT) {
        R E1[3], B1[3];
        const Local<R> L = node_local<PREC>(P, a, st_e, k);
        analytic_fields<AP_PLANE, PREC>(P, L, E1, B1);
        drive = l_add((T)E1[0], ek);
      }
      const T jk = l_add(j[k], l_mul(q[k], drive));
      j[k] = jk;
      if (k >= 1) {
        T src = jk;
        if constexpr (APT) {
          R J1[3];
          const Local<R> L = node_local<PREC>(P, a, st_j, k);
          current_plane(P, L, J1);
          src = l_sub(jk, (T)J1[0]);
        }
        e[k] = l_sub(l_sub(ek, l_mul(r, l_sub(b[k], b[k - 1]))), l_mul(dt, src));
      }
    }
    __syncthreads();
    // B^{n+1} = B^{n+1/2} - (r/2)(E_{k+1}^{n+1} - E_k^{n+1})
    for (int k = t; k < nz - 1; k += bd) b[k] = l_sub(b[k], l_mul(hr, l_sub(e[k + 1], e[k])));
  }
  // every node is written back by the thread that last wrote it
  for (int k = t; k < nz; k += bd) {
    Eg[k] = e[k];
    Bg[k] = b[k];
    Jg[k] = j[k];
  }
}

// Traditional line with the line in registers: thread t owns the C
// consecutive nodes [t C, t C + C) of E, B, J and a_k; per step only the
// values at thread boundaries move through shared memory, with two
// barriers: (1) B half step (needs E at the next thread's first node, `en`),
// publish the last B; barrier; (2) current and E update (needs B at the
// previous thread's last node), publish the first E; barrier; (3) B half
// step with the fresh `en`.  Each shared slot is written and read in
// alternate barrier intervals.  The arithmetic per node is that of
// line_kernel, so the result does not depend on C or the block size.
template <typename T, int C, int MAXT>
__global__ void __launch_bounds__(MAXT) plasma_line_reg_kernel(const __grid_constant__ LineArgs a) {
  __shared__ T s_b[kLineBlock], s_e[kLineBlock];
  const int nz = a.nz;
  const size_t off = (size_t)blockIdx.x * (size_t)nz;
  T *Eg = static_cast<T *>(a.E) + off;
  T *Bg = static_cast<T *>(a.B) + off;
  T *Jg = static_cast<T *>(a.J) + off;
  const T *W = a.wp2 ? static_cast<const T *>(a.wp2) + off : nullptr;
  const T dt = (T)a.dt;
  const T r = (T)(a.dt / a.dz);
  const T hr = (T)(0.5 * (a.dt / a.dz));
  const T wpu = (T)a.omega_p2;
  const int t = threadIdx.x;
  const int base = t * C;
  T e[C], b[C], j[C], q[C];
#pragma unroll
  for (int i = 0; i < C; ++i) {
    const int k = base + i;
    const bool in = k < nz;
    e[i] = in ? Eg[k] : T(0);
    b[i] = in ? Bg[k] : T(0);
    j[i] = in ? Jg[k] : T(0);
    q[i] = in ? l_mul(dt, W ? W[k] : wpu) : T(0);
  }
  s_e[t] = e[0];
  __syncthreads();
  T en = t + 1 < (int)blockDim.x ? s_e[t + 1] : T(0);
  for (long long n = 0; n < a.n_steps; ++n) {
#pragma unroll
    for (int i = 0; i < C; ++i) {
      const T enx = i + 1 < C ? e[i + 1] : en;
      if (base + i < nz - 1) b[i] = l_sub(b[i], l_mul(hr, l_sub(enx, e[i])));
    }
    s_b[t] = b[C - 1];
    __syncthreads();
    const T bp = t > 0 ? s_b[t - 1] : T(0);
#pragma unroll
    for (int i = 0; i < C; ++i) {
      const int k = base + i;
      if (k < nz) {
        j[i] = l_add(j[i], l_mul(q[i], e[i]));
        if (k >= 1) {
          const T bpv = i > 0 ? b[i - 1] : bp;
          e[i] = l_sub(l_sub(e[i], l_mul(r, l_sub(b[i], bpv))), l_mul(dt, j[i]));
        }
      }
    }
    s_e[t] = e[0];
    __syncthreads();
    en = t + 1 < (int)blockDim.x ? s_e[t + 1] : T(0);
#pragma unroll
    for (int i = 0; i < C; ++i) {
      const T enx = i + 1 < C ? e[i + 1] : en;
      if (base + i < nz - 1) b[i] = l_sub(b[i], l_mul(hr, l_sub(enx, e[i])));
    }
  }
#pragma unroll
  for (int i = 0; i < C; ++i) {
    const int k = base + i;
    if (k < nz) {
      Eg[k] = e[i];
      Bg[k] = b[i];
      Jg[k] = j[i];
    }
  }
}

template <typename T, int C, int MAXT>
int launch_plasma_reg(const LineArgs &a, void *stream) {
  const int block = ((a.nz + C - 1) / C + 31) / 32 * 32;
  if (block > MAXT) return AP_ERR_ARG;
  plasma_line_reg_kernel<T, C, MAXT><<<(unsigned)a.n_lines, block, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

template <typename T, int PREC, bool APT>
int launch_line_t(const Pulse<Real<PREC>> &P, const LineArgs &a, void *stream) {
  auto kern = line_kernel<T, PREC, APT>;
  const size_t per_node = 4u * sizeof(T) + ((APT && PREC == AP_FP32_PHASEFF) ? 3u * sizeof(float) : 0u);
  const size_t smem = per_node * (size_t)a.nz;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return AP_ERR_CUDA;
  int block = (a.nz + 31) / 32 * 32;
  if (block > kLineBlock) block = kLineBlock;
  kern<<<(unsigned)a.n_lines, block, smem, static_cast<cudaStream_t>(stream)>>>(P, a);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

}  // namespace

int launch_line(bool apt_mode, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                const LineArgs &a, void *stream) {
  // traditional float lines up to 8 x 768 nodes: the line in registers
  if (!apt_mode && precision != AP_FP64) {
    if (a.nz <= kLineBlock) return launch_plasma_reg<float, 1, kLineBlock>(a, stream);
    if (a.nz <= 2 * kLineBlock) return launch_plasma_reg<float, 2, kLineBlock>(a, stream);
    if (a.nz <= 4 * kLineBlock) return launch_plasma_reg<float, 4, kLineBlock>(a, stream);
    if (a.nz <= 8 * 768) return launch_plasma_reg<float, 8, 768>(a, stream);
  }
  if (precision == AP_FP64)
    return apt_mode ? launch_line_t<double, AP_FP64, true>(pd, a, stream)
                    : launch_line_t<double, AP_FP64, false>(pd, a, stream);
  return apt_mode ? launch_line_t<float, AP_FP32_PHASEFF, true>(pf, a, stream)
                  : launch_line_t<float, AP_FP32_PHASEFF, false>(pf, a, stream);
}

}  // namespace apt
