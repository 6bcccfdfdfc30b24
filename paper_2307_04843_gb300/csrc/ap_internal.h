// ap_internal.h -- structures shared by the host layer and the kernels of the
// analytic-pulse library (not part of the public C ABI in include/ap.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/ap.h"

namespace apt {

constexpr int kMaxComp = AP_MAX_COMP;
constexpr int kLgMaxP = 8;
constexpr int kLgMaxL = 8;

// Per-component constants of the flying-focus superposition (Sec. 3.3).
// Component j: zeta_j = (z - z_ref) / zR_j - zoff_j,
//   u_j = c_j q_j exp(-r^2 q_j / w0^2) e^{i omega_j phi'},  phi' = (t - t_ref) - (z - z_ref),
// with c_j = A e^{i (omega_j t_ref - k_j z_ref - Phi_j + phase0)} folded in on the host.
template <typename R>
struct Comp {
  R inv_zR;  // 1 / zR_j
  R zoff;    // (z_j - z_ref) / zR_j
  R inv_k;   // 1 / k_j (longitudinal terms)
  R c_re, c_im;
};

// Device-side description of one pulse, derived on the host in FP64 (row a1)
// and rounded once to the arithmetic type R of the push.
template <typename R>
struct Pulse {
  static constexpr bool kHasPlasma = true;  // carries the Sec. 4 plasma constants
  int32_t kind, pol, env, lon;
  int32_t lg_p, lg_al, lg_sgn, n_comp;
  int32_t sg_order, yee, plasma, pad1;
  R amp;            // amplitude coefficient A of the profile
  R inv_vg;         // 1 / v_g
  R bratio;         // B0 / E0 (Eq. e_amp; 1 in vacuum)
  R lonE, lonB;     // v_phi / omega and c / omega: d/dz -> -i omega / v, Sec. 3.1
  R inv_w0sq;       // 1 / w0^2
  R inv_zR;         // 1 / z_R
  R env_a, env_b;   // envelope constants (see ap_device.cuh)
  R px_re, px_im, py_re, py_im;  // polarisation vector p
  // Laguerre three-term recurrence (k+1) L_{k+1} = (2k+1+a-s) L_k - (k+a) L_{k-1}
  // as L_{k+1} = (lg_r[0][k] - lg_r[1][k] s) L_k - lg_r[2][k] L_{k-1}, for
  // a = |l| (rows 0-2) and a = |l| + 1 (rows 3-5, the derivative
  // dL_p^a/ds = -L_{p-1}^{a+1})
  R lg_r[6][kLgMaxP];
  R lg_pref;                     // (sqrt(2) / w0)^{|l|}
  R lg_alf;                      // |l| as a number
  R a0, inv_w0, amp_unit;        // a0, 1/w0 and amp / a0 (adjoint: d/da0, d/dw0)
  R beta_f, inv_1mb;             // closed-form flying focus: v_f / c and 1 / (1 - beta_f)
  R adv_xy;                      // 1, or 0 for 1D-3V sets (transverse position held)
  // plane wave in a linear plasma (Sec. 4): 1 - v_phi/v_g (weight of B's
  // finite-duration terms, Eq. b_corr_t), J1 amplitude omega_p^2 zeta/omega
  // (Eq. j1), 1/omega, and the constants of the envelope's logarithmic
  // derivatives (see envelope_logd)
  R fdc, jamp, inv_w, lg_c1, lg_c2;
  // carrier phase psi = omega (t - t_f) - k (z - z_f) + phase0 (double, host-exact)
  double omega, k, t_f, z_f, phase0;
  // float-float copies for AP_FP32_PHASEFF
  float k_hi, k_lo, zf_hi, zf_lo;
  // flying focus: omega_j = ff_w + j ff_dw (vacuum k_j = omega_j), with
  // float-float copies for AP_FP32_PHASEFF
  double ff_w, ff_dw;
  float ffw_hi, ffw_lo, ffd_hi, ffd_lo;
  Comp<R> comp[kMaxComp];
};

// Grid view passed to kernels (device pointers, caller-owned).
struct GridView {
  const float *f[6];
  const float4 *packed;   // node-interleaved [nz][ny][nx][2] float4, or null
  const float4 *cells;    // per-cell trilinear coefficients [nz-1][ny-1][nx-1][12] float4, or null
  int nx, ny, nz;
  float lo[3], inv_d[3];  // node spacing d = (hi - lo)/(n - 1)
  double lo_d[3], inv_d_d[3];
  float off[3];           // -lo / d: grid units u = x inv_d + off
  double off_d[3];
  float top[3], top2[3];  // n - 1 and n - 2 as floats (no per-step conversion)
};

// Diagnostics view.
struct DiagView {
  double *lf;            // [n_steps] or null
  uint32_t *hist;        // [bins] or null
  int bins;
  double hist_lo, hist_scale;
  double *set_sum;       // [n_sets] or null
};

struct LaunchShape {
  int block;
  int blocks_per_sm;
  int grid_cache;  // 0: cell in shared memory, 1: in registers (AP_PACK_CELLS only)
  int pairs;       // float-float pushes: 1 = two particles per thread (packed arithmetic)
  int tile;        // batched launch: particles per tile (0: the block's particles)
};

// Host-side launchers implemented in the per-kind translation units.
struct PushArgs {
  double *x, *y, *z;
  void *ux, *uy, *uz;
  long long n;
  double t0, dt;
  long long n_steps;
  int grid_on;
  GridView grid;
  DiagView diag;
  int *status;
  int sm_count;
  LaunchShape shape;
};

struct BatchArgs {
  PushArgs base;
  const long long *set_offsets;  // device [n_sets + 1]
  int n_sets;
  unsigned int *tile_counter;    // device scratch
  int tile;                      // particles per tile
};

struct EvalArgs {
  const double *xyzt;
  long long n;
  double *EB;
  int *status;
};

// Staggered-node evaluation (ap_eval_nodes).  comp[0..n_comp) lists the
// components present; lo and d also as float-float pairs for the
// float-float arithmetic.
struct NodeArgs {
  void *f[6];
  int nx, ny, nz;
  int f64, accumulate;
  int comp[6], n_comp;
  double lo[3], d[3];
  float lo_hi[3], lo_lo[3], d_hi[3], d_lo[3];
  double t;
  int sm_count;
  int current;  // 1: the analytic current J1 into f[0..2] (plane waves)
};

// 1-D lines with a linear cold-plasma current (ap_line.cu): the traditional
// line, or the split line with the analytic E1 and J1 of a plane-wave pulse.
struct LineArgs {
  void *E, *B, *J;
  const void *wp2;       // [n_lines][nz] or null (uniform omega_p2)
  int nz, n_lines;
  double dz, dt, omega_p2, z0, t0;
  float z0_hi, z0_lo, dz_hi, dz_lo;  // float-float node positions (AP_FP32_PHASEFF)
  long long n_steps;
};
int launch_line(bool apt, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                const LineArgs &a, void *stream);

// One launcher per pulse kind; precision selects the template instance.
// `pulse_d` / `pulse_f` are host copies; `dpulse_*` device copies (batched).
int launch_push(int kind, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                const PushArgs &a, void *stream);
int launch_eval(int kind, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                const EvalArgs &a, void *stream);
int launch_batch(int kind, int precision, const Pulse<double> *dpd, const Pulse<float> *dpf,
                 const BatchArgs &a, void *stream);
int launch_nodes(int kind, int precision, const Pulse<double> &pd, const Pulse<float> &pf,
                 const NodeArgs &a, void *stream);

// per-kind entry points (ap_push_<kind>.cu)
#define APT_DECLARE_KIND(K)                                                                       \
  int launch_push_##K(int precision, const Pulse<double> &pd, const Pulse<float> &pf,             \
                      const PushArgs &a, void *stream);                                           \
  int launch_eval_##K(int precision, const Pulse<double> &pd, const Pulse<float> &pf,             \
                      const EvalArgs &a, void *stream);                                           \
  int launch_batch_##K(int precision, const Pulse<double> *dpd, const Pulse<float> *dpf,          \
                       const BatchArgs &a, void *stream);                                         \
  int launch_nodes_##K(int precision, const Pulse<double> &pd, const Pulse<float> &pf,            \
                       const NodeArgs &a, void *stream);
APT_DECLARE_KIND(plane)
APT_DECLARE_KIND(gauss)
APT_DECLARE_KIND(lg)
APT_DECLARE_KIND(flying)
APT_DECLARE_KIND(flyingcf)
#undef APT_DECLARE_KIND

// The FP64 push and the adjoint read raw corners: they use f[] instead of a
// per-cell coefficient copy (AP_ERR_ARG when f[] is missing).
int drop_cell_layout(GridView &v);

// status bits written by kernels
constexpr int kStatusNonfinite = 1;

}  // namespace apt
