// ap_kernels.cuh -- kernels of the gather + push (rows a2-a12 of the hot
// path) and their launchers, instantiated once per pulse kind by
// ap_push_<kind>.cu (AP_KIND_ID / AP_KIND_NAME set before inclusion).
#pragma once

#include <type_traits>

#include "ap_pair.cuh"

namespace apt {

// Steps per chunk of the per-warp step table (float-float variant): one
// entry per lane.
constexpr int kStepChunk = 32;

// Dynamic shared memory of the push kernels, per block of T threads: the
// per-warp step tables (16 B per thread), then for the float grid kernels the
// cell-cache slots (16 slots x 16 B per thread).
__host__ __device__ constexpr size_t step_table_bytes(int threads) { return 16u * (size_t)threads; }
__host__ __device__ constexpr size_t grid_slot_bytes(int threads) { return 256u * (size_t)threads; }

// Grid modes of the push kernels: no grid, corner values (component arrays
// or the node-interleaved copy), per-cell coefficients (float kernels only).
constexpr int kGridNone = 0;
constexpr int kGridNodes = 1;
constexpr int kGridCells = 2;
constexpr int kGridCellsReg = 3;  // per-cell coefficients cached in registers
constexpr int kGridCellsMix = 4;  // two particles per thread: the first's cell in registers,
                                  // the second's in shared memory

// Grid cell cache of a variant: registers for double, shared memory for float.
template <int PREC, int GRID>
struct CacheOf {
  using type = GridCache<Real<PREC>>;
};
template <>
struct CacheOf<AP_FP32_PHASE64, kGridNodes> {
  using type = GridSlots;
};
template <>
struct CacheOf<AP_FP32_PHASEFF, kGridNodes> {
  using type = GridSlots;
};
template <>
struct CacheOf<AP_FP32_PHASE64, kGridCells> {
  using type = CellSlots;
};
template <>
struct CacheOf<AP_FP32_PHASEFF, kGridCells> {
  using type = CellSlots;
};
template <>
struct CacheOf<AP_FP32_PHASE64, kGridCellsReg> {
  using type = CellRegs;
};
template <>
struct CacheOf<AP_FP32_PHASEFF, kGridCellsReg> {
  using type = CellRegs;
};

// shared-memory bytes of the cell cache per block of T threads carrying NP
// particles each
template <int PREC, int GRID, int NP = 1>
__host__ __device__ constexpr size_t grid_cache_bytes(int threads) {
  return PREC == AP_FP64 || GRID == kGridNone || GRID == kGridCellsReg ? 0
         : GRID == kGridCells                                         ? 12u * kCellSlotStride * NP
         : GRID == kGridCellsMix                                      ? 12u * kCellSlotStride
                                                                      : grid_slot_bytes(threads);
}

// One particle through n_steps fused steps: load (a2), per step the local
// coordinates and phase (a3), envelope and profile (a4-a7), grid gather
// (a8), Boris and position (a9), light-front diagnostic (a10); then store
// (a11).  Every lane of a warp calls this together: the float-float variant
// tabulates the per-step phase base C_n and time T_n for its warp in shared
// memory, 32 steps at a time (one entry per lane, __syncwarp only, so warps
// never wait for each other).  `valid` is false for padding threads, which
// run the loop on a dummy particle so that warp operations see every lane.
// Returns the final gamma (double) of a valid particle, 0 otherwise.
template <int KIND, int PREC, int GRID>
__device__ __forceinline__ double push_one(const Pulse<Real<PREC>> &P, const PushArgs &a,
                                           long long i, bool valid, StepFF *s_steps,
                                           void *slots) {
  using R = Real<PREC>;
  double X = 0.0, Y = 0.0, Z = 0.0;
  R u[3] = {R(0), R(0), R(0)};
  if (valid) {
    X = a.x[i];
    Y = a.y[i];
    Z = a.z[i];
    const R *ux = static_cast<const R *>(a.ux);
    const R *uy = static_cast<const R *>(a.uy);
    const R *uz = static_cast<const R *>(a.uz);
    u[0] = ux[i];
    u[1] = uy[i];
    u[2] = uz[i];
  }
  Pos<PREC> pos;
  pos.load(X, Y, Z);
  TimeBase<PREC> tb;
  tb.init(P, a.t0, a.dt);
  const R dtR = (R)a.dt;
  const R dtxy = dtR * P.adv_xy;
  const R h0 = R(1) / rsqrt_r(fma(u[0], u[0], fma(u[1], u[1], fma(u[2], u[2], R(1))))) - u[2];
  typename CacheOf<PREC, GRID>::type gc;
  if constexpr (GRID && !std::is_same<R, double>::value) grid_slots_init(gc, slots);
  else grid_cache_reset(gc);
  double *lf = a.diag.lf;
  StepFF *wsteps = s_steps + (threadIdx.x >> 5) * kStepChunk;
  const int lane = threadIdx.x & 31;
  // the step loop, compiled twice: with the per-step light-front diagnostic
  // and without it (its test would otherwise cost every step an issue slot)
  auto steps = [&](auto with_lf) {
    constexpr bool LF = decltype(with_lf)::value;
    for (long long s0 = 0; s0 < a.n_steps; s0 += kStepChunk) {
      const int cnt = (int)(a.n_steps - s0 < kStepChunk ? a.n_steps - s0 : kStepChunk);
      if constexpr (PREC == AP_FP32_PHASEFF) {
        __syncwarp();  // no lane still reads the previous chunk
        if (lane < cnt) wsteps[lane] = tb.at(s0 + lane);
        __syncwarp();
      }
      for (int k = 0; k < cnt; ++k) {
        typename TimeBase<PREC>::Step st;
        if constexpr (PREC == AP_FP32_PHASEFF) st = wsteps[k];
        else st = tb.at(s0 + k);
        Local<R> L = local_coords<PREC>(P, st, pos);
        if constexpr (GRID) grid_fetch(a.grid, gc, L.x, L.y, pos.zr());
        R E[3], B[3];
        analytic_fields<KIND, PREC>(P, L, E, B);
        if constexpr (GRID) grid_eval(gc, E, B);
        R ig = boris(u, E, B, dtR);
        pos.advance(u[0] * ig, u[1] * ig, u[2] * ig, dtxy, dtR);
        if constexpr (LF) {
          R dev = valid ? fabs((R(1) / ig - u[2]) - h0) : R(0);
          warp_max_to(lf + s0 + k, dev, 0xffffffffu);
        }
      }
    }
  };
  if (lf) steps(std::true_type{});
  else steps(std::false_type{});
  if (!valid) return 0.0;
  pos.store(a.x + i, a.y + i, a.z + i);
  R *ux = static_cast<R *>(a.ux);
  R *uy = static_cast<R *>(a.uy);
  R *uz = static_cast<R *>(a.uz);
  ux[i] = u[0];
  uy[i] = u[1];
  uz[i] = u[2];
  const double dx = (double)u[0], dy = (double)u[1], dz = (double)u[2];
  if (!all_finite(a.x[i], a.y[i], a.z[i], dx, dy, dz)) atomicOr(a.status, kStatusNonfinite);
  // gamma in double from the stored momentum, fixed operation order
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz)),
                              1.0));
}

// Two particles per thread (float-float variant, grid none or per-cell
// coefficients in registers): particle i0 rides in the low half and i1 in the
// high half of every packed value (ap_pair.cuh), so each FP32 instruction of
// the local coordinates, the field, the Boris step and the position update
// serves both.  The steps and their order are those of push_one; each
// particle keeps its own grid cell (its refetch is its own warp-uniform
// branch) and the cell is evaluated with packed FMA over component pairs.
// `v0`, `v1` are false for padding particles.  g receives the final gammas.
// The block's pre-broadcast grid constants for grid_fetch2 (written by the
// first four threads; the caller synchronises the block before use).
__device__ __forceinline__ void grid_pair_consts(const GridView &g, float4 *gk) {
  if (threadIdx.x < 3) {
    const int ax = threadIdx.x;
    gk[ax] = make_float4(g.inv_d[ax], g.inv_d[ax], g.off[ax], g.off[ax]);
  } else if (threadIdx.x == 3) {
    gk[3] = make_float4(0.5f, 0.5f, 0.0f, 0.0f);
  }
}

template <int KIND, int GRID>
__device__ __forceinline__ void push_two(const Pulse<float> &P, const PushArgs &a, long long i0,
                                         long long i1, bool v0, bool v1, StepFF *s_steps,
                                         void *slots, const float4 *gk, double g[2]) {
  static_assert(GRID == kGridNone || GRID == kGridCells || GRID == kGridCellsReg ||
                    GRID == kGridCellsMix,
                "two-particle grid modes");
  double X[2] = {0.0, 0.0}, Y[2] = {0.0, 0.0}, Z[2] = {0.0, 0.0};
  float ua[3] = {0.0f, 0.0f, 0.0f}, ub[3] = {0.0f, 0.0f, 0.0f};
  {
    const float *ux = static_cast<const float *>(a.ux);
    const float *uy = static_cast<const float *>(a.uy);
    const float *uz = static_cast<const float *>(a.uz);
    if (v0) {
      X[0] = a.x[i0]; Y[0] = a.y[i0]; Z[0] = a.z[i0];
      ua[0] = ux[i0]; ua[1] = uy[i0]; ua[2] = uz[i0];
    }
    if (v1) {
      X[1] = a.x[i1]; Y[1] = a.y[i1]; Z[1] = a.z[i1];
      ub[0] = ux[i1]; ub[1] = uy[i1]; ub[2] = uz[i1];
    }
  }
  F2 u[3] = {F2(ua[0], ub[0]), F2(ua[1], ub[1]), F2(ua[2], ub[2])};
  Pos2 pos;
  pos.load(X, Y, Z, P.z_f);
  TimeBase<AP_FP32_PHASEFF> tb;
  tb.init(P, a.t0, a.dt);
  const float dts = (float)a.dt;
  const F2 dtR = dts, dtxy = dts * P.adv_xy;
  // light-front reference h0 = gamma - u_z on entry, per particle as in push_one
  const float h0a = 1.0f / rsqrt_r(fmaf(ua[0], ua[0], fmaf(ua[1], ua[1], fmaf(ua[2], ua[2], 1.0f)))) - ua[2];
  const float h0b = 1.0f / rsqrt_r(fmaf(ub[0], ub[0], fmaf(ub[1], ub[1], fmaf(ub[2], ub[2], 1.0f)))) - ub[2];
  // cell caches: registers, or two regions of the block's shared slots (the
  // second particle's 12 slots per thread after the first's)
  using CacheA = typename std::conditional<GRID == kGridCells, CellSlots, CellRegs>::type;
  using CacheB = typename std::conditional<GRID == kGridCellsReg, CellRegs, CellSlots>::type;
  CacheA gca;
  CacheB gcb;
  if constexpr (GRID == kGridCellsMix) {
    grid_slots_init(gca, nullptr);
    grid_slots_init(gcb, slots);
  } else if constexpr (GRID != kGridNone) {
    grid_slots_init(gca, slots);
    grid_slots_init(gcb, static_cast<unsigned char *>(slots) + 12u * kCellSlotStride);
  }
  double *lf = a.diag.lf;
  StepFF *wsteps = s_steps + (threadIdx.x >> 5) * kStepChunk;
  const int lane = threadIdx.x & 31;
  auto steps = [&](auto with_lf) {
    constexpr bool LF = decltype(with_lf)::value;
    for (long long s0 = 0; s0 < a.n_steps; s0 += kStepChunk) {
      const int cnt = (int)(a.n_steps - s0 < kStepChunk ? a.n_steps - s0 : kStepChunk);
      __syncwarp();  // no lane still reads the previous chunk
      if (lane < cnt) wsteps[lane] = tb.at(s0 + lane);
      __syncwarp();
#pragma unroll 2
      for (int k = 0; k < cnt; ++k) {
        const StepFF st = wsteps[k];
        const Local<F2> L = local_coords2(P, st, pos);
        if constexpr (GRID != kGridNone)
          grid_fetch2(a.grid, gca, gcb, L.x, L.y, pos.zr(P.zf_hi, P.zf_lo), gk);
        F2 E[3], B[3];
        analytic_fields<KIND, AP_FP32_PHASEFF, F2>(P, L, E, B);
        if constexpr (GRID != kGridNone) {
          if constexpr (GRID == kGridCells || GRID == kGridCellsMix)
            cp_async_wait_all();  // this thread's copies landed
          float oa[6], ob[6];
          grid_values(gca, oa);
          grid_values(gcb, ob);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            E[c].x += oa[c]; E[c].y += ob[c];
            B[c].x += oa[c + 3]; B[c].y += ob[c + 3];
          }
        }
        const F2 ig = boris(u, E, B, dtR);
        pos.advance(u[0] * ig, u[1] * ig, u[2] * ig, dtxy, dtR);
        if constexpr (LF) {
          const float da = v0 ? fabsf((1.0f / ig.x - u[2].x) - h0a) : 0.0f;
          const float db = v1 ? fabsf((1.0f / ig.y - u[2].y) - h0b) : 0.0f;
          warp_max_to(lf + s0 + k, fmaxf(da, db), 0xffffffffu);
        }
      }
    }
  };
  if (lf) steps(std::true_type{});
  else steps(std::false_type{});
  const long long idx[2] = {i0, i1};
  const bool val[2] = {v0, v1};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    g[h] = 0.0;
    if (!val[h]) continue;
    const long long i = idx[h];
    const FF px{h ? pos.x.hi.y : pos.x.hi.x, h ? pos.x.lo.y : pos.x.lo.x};
    const FF py{h ? pos.y.hi.y : pos.y.hi.x, h ? pos.y.lo.y : pos.y.lo.x};
    const FF pz{h ? pos.dz.hi.y : pos.dz.hi.x, h ? pos.dz.lo.y : pos.dz.lo.x};
    a.x[i] = (double)px.hi + (double)px.lo;
    a.y[i] = (double)py.hi + (double)py.lo;
    a.z[i] = ((double)pz.hi + (double)pz.lo) + P.z_f;
    const float fu[3] = {h ? u[0].y : u[0].x, h ? u[1].y : u[1].x, h ? u[2].y : u[2].x};
    static_cast<float *>(a.ux)[i] = fu[0];
    static_cast<float *>(a.uy)[i] = fu[1];
    static_cast<float *>(a.uz)[i] = fu[2];
    const double dx = (double)fu[0], dy = (double)fu[1], dz = (double)fu[2];
    if (!all_finite(a.x[i], a.y[i], a.z[i], dx, dy, dz)) atomicOr(a.status, kStatusNonfinite);
    g[h] = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                          __dmul_rn(dz, dz)),
                                1.0));
  }
}

__device__ __forceinline__ void hist_add(uint32_t *s_hist, const DiagView &d, double g) {
  if (!isfinite(g)) return;
  double f = floor(__dmul_rn(__dsub_rn(g, d.hist_lo), d.hist_scale));
  int b = f < 0.0 ? 0 : (f > (double)(d.bins - 1) ? d.bins - 1 : (int)f);
  atomicAdd(&s_hist[b], 1u);
}

// block sum of a double; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double *s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; ++k) r += s_red[k];
  return r;
}

// Plain launch: a grid-stride loop over block-sized chunks of particles (the
// trip count is uniform across the block), one particle per thread, every
// step fused.  Dynamic shared memory: step tables, grid slots (float grid
// kernels), then the histogram (hist_off bytes in).
template <int KIND, int PREC, int GRID, int NP = 1>
__device__ __forceinline__ void push_body(const Pulse<Real<PREC>> &P, const PushArgs &a, unsigned hist_off) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ double s_red[32];
  StepFF *s_steps = reinterpret_cast<StepFF *>(s_dyn);
  void *slots = s_dyn + step_table_bytes(blockDim.x);
  uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_dyn + hist_off);
  const bool hist = a.diag.hist != nullptr;
  if (hist) {
    for (int b = threadIdx.x; b < a.diag.bins; b += blockDim.x) s_hist[b] = 0u;
    __syncthreads();
  }
  __shared__ float4 s_gridk[4];
  if constexpr (NP == 2) {
    grid_pair_consts(a.grid, s_gridk);
    __syncthreads();
  }
  double acc = 0.0;
  // NP particles per thread: a block covers NP * blockDim.x consecutive
  // particles, thread t the ones at t and t + blockDim.x (coalesced)
  const long long stride = (long long)NP * gridDim.x * blockDim.x;
  for (long long base = (long long)NP * blockIdx.x * blockDim.x; base < a.n; base += stride) {
    const long long i = base + threadIdx.x;
    if constexpr (NP == 2) {
      const long long i1 = i + blockDim.x;
      double g[2];
      push_two<KIND, GRID>(P, a, i, i1, i < a.n, i1 < a.n, s_steps, slots, s_gridk, g);
      if (i < a.n) {
        acc += g[0];
        if (hist) hist_add(s_hist, a.diag, g[0]);
      }
      if (i1 < a.n) {
        acc += g[1];
        if (hist) hist_add(s_hist, a.diag, g[1]);
      }
    } else {
      const bool valid = i < a.n;
      double g = push_one<KIND, PREC, GRID>(P, a, i, valid, s_steps, slots);
      if (valid) {
        acc += g;
        if (hist) hist_add(s_hist, a.diag, g);
      }
    }
  }
  if (a.diag.set_sum) {
    double t = block_sum(acc, s_red);
    if (threadIdx.x == 0) atomicAdd(a.diag.set_sum, t);
  }
  if (hist) {
    __syncthreads();
    for (int b = threadIdx.x; b < a.diag.bins; b += blockDim.x)
      if (s_hist[b]) atomicAdd(&a.diag.hist[b], s_hist[b]);
  }
}

// Two entries for the same body.  The per-cell coefficient variants name a
// residency target (3 blocks of 256 with the cell in shared memory, 2 with
// it in registers); the others keep the compiler's own register choice (an
// explicit minimum of one block lets it spend registers freely, which cost
// the flying-focus kernel 7 % through lost occupancy).
template <int KIND, int PREC, int GRID>
__global__ void __launch_bounds__(256)
    push_kernel(const __grid_constant__ Pulse<Real<PREC>> P, const __grid_constant__ PushArgs a,
                unsigned hist_off) {
  push_body<KIND, PREC, GRID>(P, a, hist_off);
}

template <int KIND, int PREC, int GRID>
__global__ void __launch_bounds__(256, GRID == kGridCells ? 3 : 2)
    push_kernel_cells(const __grid_constant__ Pulse<Real<PREC>> P, const __grid_constant__ PushArgs a,
                      unsigned hist_off) {
  push_body<KIND, PREC, GRID>(P, a, hist_off);
}

// Two particles per thread (AP_FP32_PHASEFF; no grid, or per-cell
// coefficients cached in shared memory or in registers).
template <int KIND, int GRID>
__global__ void __launch_bounds__(256)
    push_kernel_pair(const __grid_constant__ Pulse<float> P, const __grid_constant__ PushArgs a,
                     unsigned hist_off) {
  push_body<KIND, AP_FP32_PHASEFF, GRID, 2>(P, a, hist_off);
}
// cells in shared memory: 2 resident blocks of 256 (384 B of slots per thread)
template <int KIND>
__global__ void __launch_bounds__(256, 2)
    push_kernel_pair_smem(const __grid_constant__ Pulse<float> P, const __grid_constant__ PushArgs a,
                          unsigned hist_off) {
  push_body<KIND, AP_FP32_PHASEFF, kGridCells, 2>(P, a, hist_off);
}
// first cell in registers, second in shared memory: 2 resident blocks of 256
// (128 registers, 192 B of slots per thread)
template <int KIND>
__global__ void __launch_bounds__(256, 2)
    push_kernel_pair_mix(const __grid_constant__ Pulse<float> P, const __grid_constant__ PushArgs a,
                         unsigned hist_off) {
  push_body<KIND, AP_FP32_PHASEFF, kGridCellsMix, 2>(P, a, hist_off);
}


template <int KIND, int PREC, int GRID>
constexpr auto push_entry() {
  if constexpr (GRID == kGridCells || GRID == kGridCellsReg) return push_kernel_cells<KIND, PREC, GRID>;
  else return push_kernel<KIND, PREC, GRID>;
}

// Batched persistent launch (row a12): blocks pop fixed-size tiles of
// (set, particles) from a global counter until the tile count is reached;
// each set's pulse is copied to shared memory; the loop is bounded by the
// tile count and no block waits on another.
// Dynamic shared memory: step tables, grid slots (float grid kernels), then
// the [n_sets + 1] tile prefix (prefix_off bytes in).
template <int KIND, int PREC, int GRID, int NP>
__device__ __forceinline__ void batch_body(const Pulse<Real<PREC>> *__restrict__ sets,
                                           const BatchArgs &ba, unsigned prefix_off) {
  using R = Real<PREC>;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ double s_red[32];
  __shared__ long long s_tile;
  __shared__ int s_set;
  StepFF *s_steps = reinterpret_cast<StepFF *>(s_dyn);
  void *slots = s_dyn + step_table_bytes(blockDim.x);
  long long *s_prefix = reinterpret_cast<long long *>(s_dyn + prefix_off);
  __shared__ __align__(16) unsigned char s_pulse_raw[sizeof(Pulse<R>)];
  Pulse<R> &sp = *reinterpret_cast<Pulse<R> *>(s_pulse_raw);
  const PushArgs &a = ba.base;
  const int T = ba.tile;
  __shared__ float4 s_gridk[4];
  if constexpr (NP == 2) grid_pair_consts(a.grid, s_gridk);  // the prefix's barrier follows
  // tile prefix over sets: tiles of set s = ceil(N_s / T)
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int s = 0; s < ba.n_sets; ++s) {
      s_prefix[s] = acc;
      long long ns = ba.set_offsets[s + 1] - ba.set_offsets[s];
      if (ns < 0) ns = 0;  // malformed offsets: no tiles (particles are bounds-checked below)
      acc += (ns + T - 1) / T;
    }
    s_prefix[ba.n_sets] = acc;
    s_set = -1;
  }
  __syncthreads();
  const long long total = s_prefix[ba.n_sets];
  // per-set pulse size copied to shared memory (flying focus: only n_comp components)
  for (;;) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(ba.tile_counter, 1u);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= total) break;
    // set of this tile: last s with prefix[s] <= tile (binary search)
    int lo = 0, hi = ba.n_sets;
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
    const long long first = ba.set_offsets[set] + (tile - s_prefix[set]) * T;
    const long long end_set = ba.set_offsets[set + 1];
    double acc = 0.0;
    // T is a multiple of NP * blockDim.x: every thread runs the same trip count
    for (int k = threadIdx.x; k < T; k += NP * blockDim.x) {
      const long long i = first + k;
      const bool valid = i >= 0 && i < end_set && i < a.n;
      if constexpr (NP == 2) {
        const long long i1 = i + blockDim.x;
        const bool valid1 = i1 >= 0 && i1 < end_set && i1 < a.n;
        double g[2];
        push_two<KIND, GRID>(sp, a, i, i1, valid, valid1, s_steps, slots, s_gridk, g);
        if (valid) acc += g[0];
        if (valid1) acc += g[1];
      } else {
        double g = push_one<KIND, PREC, GRID>(sp, a, i, valid, s_steps, slots);
        if (valid) acc += g;
      }
    }
    if (a.diag.set_sum) {
      double t = block_sum(acc, s_red);
      if (threadIdx.x == 0) atomicAdd(a.diag.set_sum + set, t);
    }
    __syncthreads();
  }
}

template <int KIND, int PREC, int GRID, int NP = 1>
__global__ void __launch_bounds__(256) batch_kernel(const Pulse<Real<PREC>> *__restrict__ sets,
                                                    const __grid_constant__ BatchArgs ba,
                                                    unsigned prefix_off) {
  batch_body<KIND, PREC, GRID, NP>(sets, ba, prefix_off);
}
// two particles per thread with one or both cells in shared memory: 2 blocks
// of 256
template <int KIND, int GRID>
__global__ void __launch_bounds__(256, 2)
    batch_kernel_pair_2b(const Pulse<float> *__restrict__ sets, const __grid_constant__ BatchArgs ba,
                         unsigned prefix_off) {
  batch_body<KIND, AP_FP32_PHASEFF, GRID, 2>(sets, ba, prefix_off);
}

// Field evaluation hook: one point per thread, the push's own code path at
// step 0 of a time base starting at the point's t.
template <int KIND, int PREC>
__global__ void __launch_bounds__(256) eval_kernel(const __grid_constant__ Pulse<Real<PREC>> P,
                                                   const __grid_constant__ EvalArgs a) {
  using R = Real<PREC>;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double x = a.xyzt[i], y = a.xyzt[a.n + i], z = a.xyzt[2 * a.n + i],
               t = a.xyzt[3 * a.n + i];
  Pos<PREC> pos;
  pos.load(x, y, z);
  TimeBase<PREC> tb;
  tb.init(P, t, 0.0);
  Local<R> L = local_coords<PREC>(P, tb.at(0), pos);
  R E[3], B[3];
  analytic_fields<KIND, PREC>(P, L, E, B);
  for (int c = 0; c < 3; ++c) {
    a.EB[(long long)c * a.n + i] = (double)E[c];
    a.EB[(long long)(c + 3) * a.n + i] = (double)B[c];
  }
}

// Analytic fields on the staggered nodes of a Yee grid (ap_eval_nodes).
// blockIdx.y picks one present component c; threads stride over the nodes,
// x fastest, so every store is coalesced.  Component c is sampled at
// lo + (idx + off_c) d with the Yee offsets off = Ex (1/2,0,0), Ey (0,1/2,0),
// Ez (0,0,1/2), Bx (0,1/2,1/2), By (1/2,0,1/2), Bz (1/2,1/2,0); E and B both
// at time t.  The node index advances by the fixed grid stride with carries
// (one division per thread), and in the float-float variant the node
// position is formed in float-float arithmetic, so the loop issues no
// double-precision instruction.
__device__ __forceinline__ FF node_coord_ff(float f, float lo_hi, float lo_lo, float d_hi, float d_lo) {
  FF p = two_prod(f, d_hi);
  p.lo = __fmaf_rn(f, d_lo, p.lo);
  FF s = two_sum(lo_hi, p.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(lo_lo, p.lo));
  const float hi = __fadd_rn(s.hi, s.lo);
  return {hi, __fsub_rn(s.lo, __fsub_rn(hi, s.hi))};
}

// What a node receives: the analytic E1, B1, or (plane waves, `current`)
// the analytic current J1 in place of E with B zero.
template <int KIND, int PREC>
__device__ __forceinline__ void node_values(const Pulse<Real<PREC>> &P, const Local<Real<PREC>> &L,
                                            int current, Real<PREC> E[3], Real<PREC> B[3]) {
  if constexpr (KIND == AP_PLANE) {
    if (current) {
      current_plane(P, L, E);
      B[0] = B[1] = B[2] = Real<PREC>(0);
      return;
    }
  }
  analytic_fields<KIND, PREC>(P, L, E, B);
}

template <int KIND, int PREC, typename T>
__global__ void __launch_bounds__(256) nodes_kernel(const __grid_constant__ Pulse<Real<PREC>> P,
                                                    const __grid_constant__ NodeArgs a) {
  using R = Real<PREC>;
  using W = typename std::conditional<(sizeof(T) > sizeof(R)), T, R>::type;
  const int c = a.comp[blockIdx.y];
  T *__restrict__ f = static_cast<T *>(a.f[c]);
  const float ox = (c == 0 || c == 4 || c == 5) ? 0.5f : 0.0f;
  const float oy = (c == 1 || c == 3 || c == 5) ? 0.5f : 0.0f;
  const float oz = (c == 2 || c == 3 || c == 4) ? 0.5f : 0.0f;
  const long long nxy = (long long)a.nx * a.ny;
  const long long total = nxy * a.nz;
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= total) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // node (i, j, k) of n and the stride split the same way; every index is
  // below 2^23 (checked on the host), so index + stride stays exact in float
  int k = (int)(n / nxy);
  int j = (int)((n - (long long)k * nxy) / a.nx);
  int i = (int)(n - (long long)k * nxy - (long long)j * a.nx);
  const long long sk64 = stride / nxy;
  const int sj = (int)((stride - sk64 * nxy) / a.nx);
  const int si = (int)(stride - sk64 * nxy - (long long)sj * a.nx);
  const int sk = (int)(sk64 < (1 << 30) ? sk64 : (1 << 30));
  // float copies of the indices, advanced alongside (int -> float
  // conversions run on the double-precision pipe)
  float fi = (float)i, fj = (float)j, fk = (float)k;
  const float fsi = (float)si, fsj = (float)sj, fsk = (float)sk;
  const float fnx = (float)a.nx, fny = (float)a.ny;
  TimeBase<PREC> tb;
  tb.init(P, a.t, 0.0);
  const typename TimeBase<PREC>::Step st = tb.at(0);
  for (; n < total; n += stride) {
    Pos<PREC> pos;
    if constexpr (PREC == AP_FP32_PHASEFF) {
      // the transverse coordinates enter the fields in float; only z feeds
      // the carrier phase and needs the float-float sum
      pos.x = FF{fmaf(fi + ox, a.d_hi[0], a.lo_hi[0]), 0.0f};
      pos.y = FF{fmaf(fj + oy, a.d_hi[1], a.lo_hi[1]), 0.0f};
      pos.z = node_coord_ff(fk + oz, a.lo_hi[2], a.lo_lo[2], a.d_hi[2], a.d_lo[2]);
    } else {
      pos.load(fma((double)i + ox, a.d[0], a.lo[0]), fma((double)j + oy, a.d[1], a.lo[1]),
               fma((double)k + oz, a.d[2], a.lo[2]));
    }
    Local<R> L = local_coords<PREC>(P, st, pos);
    R E[3], B[3];
    node_values<KIND, PREC>(P, L, a.current, E, B);
    const R v = c == 0 ? E[0] : c == 1 ? E[1] : c == 2 ? E[2] : c == 3 ? B[0] : c == 4 ? B[1] : B[2];
    f[n] = a.accumulate ? (T)((W)f[n] + (W)v) : (T)v;
    // advance (i, j, k) by the stride (k only grows until the loop ends)
    i += si;
    fi += fsi;
    int cj = 0;
    if (i >= a.nx) { i -= a.nx; fi -= fnx; cj = 1; }
    j += sj + cj;
    fj += fsj + (cj ? 1.0f : 0.0f);
    int ck = 0;
    if (j >= a.ny) { j -= a.ny; fj -= fny; ck = 1; }
    k = min(k + sk + ck, 1 << 30);
    fk += fsk + (ck ? 1.0f : 0.0f);
  }
}

// ------------------------------------------------------------ launchers

template <typename K>
inline int occupancy_blocks(K kernel, int block, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

// dynamic shared memory before the kernel-specific tail (histogram / prefix)
template <int PREC, int GRID, int NP = 1>
inline size_t push_smem_head(int block) {
  return step_table_bytes(block) + grid_cache_bytes<PREC, GRID, NP>(block);
}

template <typename K>
inline int set_smem(K kern, size_t smem) {
  if (smem <= 48 * 1024) return AP_OK;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                 cudaSuccess
             ? AP_OK
             : AP_ERR_CUDA;
}

template <int KIND, int PREC, int GRID>
int launch_push_t(const Pulse<Real<PREC>> &P, const PushArgs &a, void *stream) {
  auto kern = push_entry<KIND, PREC, GRID>();
  const int block = a.shape.block;
  const size_t head = push_smem_head<PREC, GRID>(block);
  const size_t smem = head + (a.diag.hist ? (size_t)a.diag.bins * sizeof(uint32_t) : 0);
  if (set_smem(kern, smem) != AP_OK) return AP_ERR_CUDA;
  const long long npad = (a.n + 31) & ~31LL;
  long long want = (npad + block - 1) / block;
  int per_sm = a.shape.blocks_per_sm > 0 ? a.shape.blocks_per_sm : occupancy_blocks(kern, block, smem);
  long long cap = (long long)a.sm_count * per_sm;
  int grid = (int)(want < cap ? want : cap);
  if (grid < 1) grid = 1;
  kern<<<grid, block, smem, static_cast<cudaStream_t>(stream)>>>(P, a, (unsigned)head);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

// the two-particle kernel of a grid mode (each with its residency target)
template <int KIND, int GRID>
constexpr auto push_pair_entry() {
  if constexpr (GRID == kGridCells) return push_kernel_pair_smem<KIND>;
  else if constexpr (GRID == kGridCellsMix) return push_kernel_pair_mix<KIND>;
  else return push_kernel_pair<KIND, GRID>;
}

template <int KIND, int GRID>
int launch_push_pair_t(const Pulse<float> &P, const PushArgs &a, void *stream) {
  auto kern = push_pair_entry<KIND, GRID>();
  const int block = a.shape.block;
  const size_t head = push_smem_head<AP_FP32_PHASEFF, GRID, 2>(block);
  const size_t smem = head + (a.diag.hist ? (size_t)a.diag.bins * sizeof(uint32_t) : 0);
  if (set_smem(kern, smem) != AP_OK) return AP_ERR_CUDA;
  const long long per_block = 2LL * block;
  const long long want = (a.n + per_block - 1) / per_block;
  int per_sm = a.shape.blocks_per_sm > 0 ? a.shape.blocks_per_sm : occupancy_blocks(kern, block, smem);
  long long cap = (long long)a.sm_count * per_sm;
  int grid = (int)(want < cap ? want : cap);
  if (grid < 1) grid = 1;
  kern<<<grid, block, smem, static_cast<cudaStream_t>(stream)>>>(P, a, (unsigned)head);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

template <int KIND, int PREC>
int launch_eval_t(const Pulse<Real<PREC>> &P, const EvalArgs &a, void *stream) {
  const int block = 128;
  const long long grid = (a.n + block - 1) / block;
  eval_kernel<KIND, PREC><<<(unsigned)grid, block, 0, static_cast<cudaStream_t>(stream)>>>(P, a);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

// All requested components of every node in one thread.  The six staggered
// positions of a node share two z levels -- the whole node (Ex, Ey, Bz) and
// the half node (Ez, Bx, By) -- so the z- and t-only part of the evaluation
// (local coordinates and carrier phase, envelope, and for beams the complex
// q = 1/(1 - i zeta)) is computed once per level: the six evaluations are
// straight-line code with identical z-only inputs, which the compiler
// computes once.  Used when three or more components are requested.
template <int KIND, int PREC, typename T>
__global__ void __launch_bounds__(256) nodes_all_kernel(const __grid_constant__ Pulse<Real<PREC>> P,
                                                        const __grid_constant__ NodeArgs a) {
  using R = Real<PREC>;
  using W = typename std::conditional<(sizeof(T) > sizeof(R)), T, R>::type;
  unsigned want = 0u;  // bit c: component c requested (a register, not an indexed array)
  for (int q = 0; q < a.n_comp; ++q) want |= 1u << a.comp[q];
  const long long nxy = (long long)a.nx * a.ny;
  const long long total = nxy * a.nz;
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= total) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // node (i, j, k) of n and of the stride, advanced as in nodes_kernel (float
  // copies of the indices: no int-to-float conversion per node)
  int k = (int)(n / nxy);
  int j = (int)((n - (long long)k * nxy) / a.nx);
  int i = (int)(n - (long long)k * nxy - (long long)j * a.nx);
  const long long sk64 = stride / nxy;
  const int sj = (int)((stride - sk64 * nxy) / a.nx);
  const int si = (int)(stride - sk64 * nxy - (long long)sj * a.nx);
  const int sk = (int)(sk64 < (1 << 30) ? sk64 : (1 << 30));
  float fi = (float)i, fj = (float)j, fk = (float)k;
  const float fsi = (float)si, fsj = (float)sj, fsk = (float)sk;
  const float fnx = (float)a.nx, fny = (float)a.ny;
  TimeBase<PREC> tb;
  tb.init(P, a.t, 0.0);
  const typename TimeBase<PREC>::Step st = tb.at(0);
  for (; n < total; n += stride) {
    Local<R> Lz[2];
    R xs[2], ys[2];  // transverse coordinates at the whole and the half node
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float o = h ? 0.5f : 0.0f;
      Pos<PREC> pos;
      if constexpr (PREC == AP_FP32_PHASEFF) {
        pos.x = FF{0.0f, 0.0f};
        pos.y = FF{0.0f, 0.0f};
        pos.z = node_coord_ff(fk + o, a.lo_hi[2], a.lo_lo[2], a.d_hi[2], a.d_lo[2]);
        xs[h] = fmaf(fi + o, a.d_hi[0], a.lo_hi[0]);
        ys[h] = fmaf(fj + o, a.d_hi[1], a.lo_hi[1]);
      } else {
        pos.load(0.0, 0.0, fma((double)k + o, a.d[2], a.lo[2]));
        xs[h] = (R)fma((double)i + o, a.d[0], a.lo[0]);
        ys[h] = (R)fma((double)j + o, a.d[1], a.lo[1]);
      }
      Lz[h] = local_coords<PREC>(P, st, pos);
    }
    // component c at (x, y, z) offsets (Ex (1/2,0,0), Ey (0,1/2,0), Ez (0,0,1/2),
    // Bx (0,1/2,1/2), By (1/2,0,1/2), Bz (1/2,1/2,0))
    constexpr int kOx[6] = {1, 0, 0, 0, 1, 1}, kOy[6] = {0, 1, 0, 1, 0, 1}, kOz[6] = {0, 0, 1, 1, 1, 0};
    R v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      Local<R> L = Lz[kOz[c]];
      L.x = xs[kOx[c]];
      L.y = ys[kOy[c]];
      R E[3], B[3];
      node_values<KIND, PREC>(P, L, a.current, E, B);
      v[c] = c < 3 ? E[c] : B[c - 3];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      if (!((want >> c) & 1u)) continue;
      T *f = static_cast<T *>(a.f[c]);
      f[n] = a.accumulate ? (T)((W)f[n] + (W)v[c]) : (T)v[c];
    }
    i += si;
    fi += fsi;
    int cj = 0;
    if (i >= a.nx) { i -= a.nx; fi -= fnx; cj = 1; }
    j += sj + cj;
    fj += fsj + (cj ? 1.0f : 0.0f);
    int ck = 0;
    if (j >= a.ny) { j -= a.ny; fj -= fny; ck = 1; }
    k = min(k + sk + ck, 1 << 30);
    fk += fsk + (ck ? 1.0f : 0.0f);
  }
}

// Rows of nx >= 32 nodes, three or more components: one warp per (y, z)
// row, lane l taking the nodes x = l, l + 32, ... (coalesced stores).  The
// z/t part of the six staggered evaluations (local coordinates and carrier
// phase, envelope, q) depends only on the row's two z levels: each lane
// computes it once per row and reuses it for all its nodes, so per node only
// the position part of the six evaluations remains (straight-line code, as
// in nodes_all_kernel).
template <int KIND, int PREC, typename T>
__global__ void __launch_bounds__(256) nodes_row_kernel(const __grid_constant__ Pulse<Real<PREC>> P,
                                                        const __grid_constant__ NodeArgs a) {
  using R = Real<PREC>;
  using W = typename std::conditional<(sizeof(T) > sizeof(R)), T, R>::type;
  unsigned want = 0u;
  for (int q = 0; q < a.n_comp; ++q) want |= 1u << a.comp[q];
  const long long rows = (long long)a.ny * a.nz;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const float flane = (float)lane;
  TimeBase<PREC> tb;
  tb.init(P, a.t, 0.0);
  const typename TimeBase<PREC>::Step st = tb.at(0);
  constexpr int kOx[6] = {1, 0, 0, 0, 1, 1}, kOy[6] = {0, 1, 0, 1, 0, 1}, kOz[6] = {0, 0, 1, 1, 1, 0};
  for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const int k = (int)(r / a.ny);
    const int j = (int)(r - (long long)k * a.ny);
    Local<R> Lz[2];
    R ys[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float o = h ? 0.5f : 0.0f;
      Pos<PREC> pos;
      if constexpr (PREC == AP_FP32_PHASEFF) {
        pos.x = FF{0.0f, 0.0f};
        pos.y = FF{0.0f, 0.0f};
        pos.z = node_coord_ff((float)k + o, a.lo_hi[2], a.lo_lo[2], a.d_hi[2], a.d_lo[2]);
        ys[h] = fmaf((float)j + o, a.d_hi[1], a.lo_hi[1]);
      } else {
        pos.load(0.0, 0.0, fma((double)k + o, a.d[2], a.lo[2]));
        ys[h] = (R)fma((double)j + o, a.d[1], a.lo[1]);
      }
      Lz[h] = local_coords<PREC>(P, st, pos);
    }
    const long long base = r * a.nx;
    float fi = flane;
    for (int i = lane; i < a.nx; i += 32, fi += 32.0f) {
      R xs[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float o = h ? 0.5f : 0.0f;
        if constexpr (PREC == AP_FP32_PHASEFF) xs[h] = fmaf(fi + o, a.d_hi[0], a.lo_hi[0]);
        else xs[h] = (R)fma((double)i + o, a.d[0], a.lo[0]);
      }
      R v[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        Local<R> L = Lz[kOz[c]];
        L.x = xs[kOx[c]];
        L.y = ys[kOy[c]];
        R E[3], B[3];
        node_values<KIND, PREC>(P, L, a.current, E, B);
        v[c] = c < 3 ? E[c] : B[c - 3];
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (!((want >> c) & 1u)) continue;
        T *f = static_cast<T *>(a.f[c]) + base;
        f[i] = a.accumulate ? (T)((W)f[i] + (W)v[c]) : (T)v[c];
      }
    }
  }
}

// The row kernel with two nodes per lane and iteration (float-float, beams):
// lane l takes x = l + 64 m and l + 64 m + 32, the two halves of every packed
// value (ap_pair.cuh), so the position part of the six evaluations -- the
// only per-node work -- issues once for both nodes.  Each warp takes a
// contiguous run of rows, so the z/t part of its rows (carrier phase and
// envelope argument; for Gaussian beams also the envelope and q) is computed
// only when the z index changes, once per run of up to ny rows, instead of
// once per row.  Stores stay coalesced: the warp writes 32 consecutive
// elements for each half.
template <int KIND, typename T>
__global__ void __launch_bounds__(256) nodes_row_pair_kernel(const __grid_constant__ Pulse<float> P,
                                                             const __grid_constant__ NodeArgs a) {
  using W = typename std::conditional<(sizeof(T) > sizeof(float)), T, float>::type;
  constexpr bool kGaussZ = KIND == AP_GAUSS || KIND == AP_FLYING_CF;
  unsigned want = 0u;
  for (int q = 0; q < a.n_comp; ++q) want |= 1u << a.comp[q];
  const long long rows = (long long)a.ny * a.nz;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long per = (rows + warps - 1) / warps;
  const long long r0 = wid * per, r1 = r0 + per < rows ? r0 + per : rows;
  const float flane = (float)lane;
  TimeBase<AP_FP32_PHASEFF> tb;
  tb.init(P, a.t, 0.0);
  const StepFF st = tb.at(0);
  constexpr int kOx[6] = {1, 0, 0, 0, 1, 1}, kOy[6] = {0, 1, 0, 1, 0, 1}, kOz[6] = {0, 0, 1, 1, 1, 0};
  int kcur = -1;
  Local<F2> Lz[2];
  BeamZ<F2> Bz[2];
  // (j, k) of the run's first row by one division, then stepped row by row
  int k = (int)(r0 / a.ny);
  int j = (int)(r0 - (long long)k * a.ny);
  for (long long r = r0; r < r1; ++r, ++j) {
    if (j == a.ny) {
      j = 0;
      ++k;
    }
    if (k != kcur) {  // uniform across the warp
      kcur = k;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        Pos<AP_FP32_PHASEFF> pos;
        pos.x = FF{0.0f, 0.0f};
        pos.y = FF{0.0f, 0.0f};
        pos.z = node_coord_ff((float)k + (h ? 0.5f : 0.0f), a.lo_hi[2], a.lo_lo[2], a.d_hi[2], a.d_lo[2]);
        const Local<float> l = local_coords<AP_FP32_PHASEFF>(P, st, pos);
        if constexpr (kGaussZ) {
          const BeamZ<float> b = gauss_z<KIND == AP_FLYING_CF>(P, l);
          Bz[h] = BeamZ<F2>{Cx<F2>{F2(b.q.re), F2(b.q.im)}, F2(b.amp_mul), F2(b.l2), F2(b.psi)};
        } else {
          Lz[h] = Local<F2>{F2(l.x), F2(l.y), F2(l.dz), F2(l.psi), F2(l.eta), F2(l.T), F2(l.phi_hi),
                            F2(l.phi_lo)};
        }
      }
    }
    const float ys[2] = {fmaf((float)j, a.d_hi[1], a.lo_hi[1]), fmaf((float)j + 0.5f, a.d_hi[1], a.lo_hi[1])};
    const long long base = r * a.nx;
    float fi = flane;
    for (int i = lane; i < a.nx; i += 64, fi += 64.0f) {
      const bool second = i + 32 < a.nx;
      F2 xs[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float o = h ? 0.5f : 0.0f;
        xs[h] = fma(F2(fi + o, fi + (32.0f + o)), F2(a.d_hi[0]), F2(a.lo_hi[0]));
      }
      F2 v[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        F2 E[3], B[3];
        if constexpr (kGaussZ) {
          gauss_xy(P, Bz[kOz[c]], xs[kOx[c]], F2(ys[kOy[c]]), E, B);
        } else {
          Local<F2> L = Lz[kOz[c]];
          L.x = xs[kOx[c]];
          L.y = F2(ys[kOy[c]]);
          analytic_fields<KIND, AP_FP32_PHASEFF, F2>(P, L, E, B);
        }
        v[c] = c < 3 ? E[c] : B[c - 3];
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (!((want >> c) & 1u)) continue;
        T *f = static_cast<T *>(a.f[c]) + base;
        f[i] = a.accumulate ? (T)((W)f[i] + (W)v[c].x) : (T)v[c].x;
        if (second) f[i + 32] = a.accumulate ? (T)((W)f[i + 32] + (W)v[c].y) : (T)v[c].y;
      }
    }
  }
}

// One warp writes the value v along a row of n elements (store, or add to
// what the row holds, rounding once to T): a scalar head up to the first
// 16-byte boundary, then 16-byte vector stores, then a scalar tail.  The row
// is aligned to sizeof(T) (checked on the host), so the head is at most
// 16 / sizeof(T) - 1 elements.
template <typename T, typename W>
__device__ __forceinline__ void row_put(T *__restrict__ row, int n, W v, bool acc, int lane) {
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int kVe = 16 / (int)sizeof(T);
  int head = (int)(((16u - ((unsigned)reinterpret_cast<uintptr_t>(row) & 15u)) & 15u) / sizeof(T));
  if (head > n) head = n;
  const int nv = (n - head) / kVe;
  const int tail = head + nv * kVe;
  V *rv = reinterpret_cast<V *>(row + head);
  // two separate loops: the store path must not read the row
  if (acc) {
    if (lane < head) row[lane] = (T)((W)row[lane] + v);
    for (int i = lane; i < nv; i += 32) {
      V x = rv[i];
      if constexpr (sizeof(T) == 4) {
        x.x = (T)((W)x.x + v); x.y = (T)((W)x.y + v); x.z = (T)((W)x.z + v); x.w = (T)((W)x.w + v);
      } else {
        x.x = (T)((W)x.x + v); x.y = (T)((W)x.y + v);
      }
      rv[i] = x;
    }
    for (int i = tail + lane; i < n; i += 32) row[i] = (T)((W)row[i] + v);
  } else {
    const T vt = (T)v;
    V x;
    if constexpr (sizeof(T) == 4) x = make_float4(vt, vt, vt, vt);
    else x = make_double2(vt, vt);
    if (lane < head) row[lane] = vt;
    for (int i = lane; i < nv; i += 32) rv[i] = x;
    for (int i = tail + lane; i < n; i += 32) row[i] = vt;
  }
}

// Plane waves (Eqs. plane_func, plane_b) depend on z and t only.  A row of
// nx nodes (fixed y, z) holds two z positions: the whole node z_k (Ex, Ey,
// Bz) and the half node z_k + dz/2 (Ez, Bx, By).  One warp per row
// evaluates the field once at each position it needs (every lane computes
// the same value), then streams each requested component along its row with
// 16-byte stores, so for nx >= 32 the kernel is bound by the stores, not the
// arithmetic.
template <int PREC, typename T>
__global__ void __launch_bounds__(256) nodes_plane_kernel(const __grid_constant__ Pulse<Real<PREC>> P,
                                                          const __grid_constant__ NodeArgs a) {
  using R = Real<PREC>;
  using W = typename std::conditional<(sizeof(T) > sizeof(R)), T, R>::type;
  bool need[2] = {false, false};  // whole, half
  for (int i = 0; i < a.n_comp; ++i) {
    const int c = a.comp[i];
    if (c == 2 || c == 3 || c == 4) need[1] = true;
    else need[0] = true;
  }
  const long long rows = (long long)a.ny * a.nz;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  TimeBase<PREC> tb;
  tb.init(P, a.t, 0.0);
  const typename TimeBase<PREC>::Step st = tb.at(0);
  for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const int k = (int)(r / a.ny);
    R v[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!need[h]) continue;
      const float oz = h ? 0.5f : 0.0f;
      Pos<PREC> pos;
      if constexpr (PREC == AP_FP32_PHASEFF) {
        pos.x = FF{0.0f, 0.0f};
        pos.y = FF{0.0f, 0.0f};
        pos.z = node_coord_ff((float)k + oz, a.lo_hi[2], a.lo_lo[2], a.d_hi[2], a.d_lo[2]);
      } else {
        pos.load(0.0, 0.0, fma((double)k + oz, a.d[2], a.lo[2]));
      }
      Local<R> L = local_coords<PREC>(P, st, pos);
      R E[3], B[3];
      node_values<AP_PLANE, PREC>(P, L, a.current, E, B);
      if (h == 0) {
        v[0] = E[0];
        v[1] = E[1];
        v[5] = B[2];
      } else {
        v[2] = E[2];
        v[3] = B[0];
        v[4] = B[1];
      }
    }
    for (int i = 0; i < a.n_comp; ++i) {
      const int c = a.comp[i];
      const R val = c == 0 ? v[0] : c == 1 ? v[1] : c == 2 ? v[2] : c == 3 ? v[3] : c == 4 ? v[4] : v[5];
      row_put<T, W>(static_cast<T *>(a.f[c]) + r * a.nx, a.nx, (W)val, a.accumulate != 0, lane);
    }
  }
}

template <int KIND, int PREC>
int launch_nodes_t(const Pulse<Real<PREC>> &P, const NodeArgs &a, void *stream) {
  const long long total = (long long)a.nx * a.ny * a.nz;
  const int block = 256;
  if constexpr (KIND == AP_PLANE) {
    if (a.nx >= 32) {
      const long long rows = (long long)a.ny * a.nz;
      long long gx = (rows + 7) / 8;  // 8 warps (rows) per block, every component of a row
      const long long cap = (long long)a.sm_count * 8;
      if (gx > cap) gx = cap;
      if (gx < 1) gx = 1;
      const dim3 grid((unsigned)gx, 1u);
      cudaStream_t s = static_cast<cudaStream_t>(stream);
      if (a.f64) nodes_plane_kernel<PREC, double><<<grid, block, 0, s>>>(P, a);
      else nodes_plane_kernel<PREC, float><<<grid, block, 0, s>>>(P, a);
      return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
    }
  }
  if (a.n_comp >= 3 && a.nx >= 32) {
    const long long rows = (long long)a.ny * a.nz;
    long long gx = (rows + 7) / 8;  // 8 warps (rows) per block
    const long long cap = (long long)a.sm_count * 8;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if constexpr (PREC == AP_FP32_PHASEFF && KIND != AP_PLANE) {
      // beams in float-float arithmetic: two nodes per lane, packed; one
      // resident wave of blocks, each warp a contiguous run of rows
      if (!a.current) {
        auto kern = a.f64 ? nodes_row_pair_kernel<KIND, double> : nodes_row_pair_kernel<KIND, float>;
        long long gp = (long long)a.sm_count * occupancy_blocks(kern, block, 0);
        if (gp > (rows + 7) / 8) gp = (rows + 7) / 8;
        if (gp < 1) gp = 1;
        kern<<<(unsigned)gp, block, 0, s>>>(P, a);
        return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
      }
    }
    if (a.f64) nodes_row_kernel<KIND, PREC, double><<<(unsigned)gx, block, 0, s>>>(P, a);
    else nodes_row_kernel<KIND, PREC, float><<<(unsigned)gx, block, 0, s>>>(P, a);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
  }
  if (a.n_comp >= 3) {
    long long gx = (total + block - 1) / block;
    const long long cap = (long long)a.sm_count * 8;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (a.f64) nodes_all_kernel<KIND, PREC, double><<<(unsigned)gx, block, 0, s>>>(P, a);
    else nodes_all_kernel<KIND, PREC, float><<<(unsigned)gx, block, 0, s>>>(P, a);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
  }
  long long gx = (total + block - 1) / block;
  // enough resident threads per component to fill the GPU, then grid-stride
  long long cap = ((long long)a.sm_count * 8 + a.n_comp - 1) / a.n_comp;
  if (gx > cap) gx = cap;
  if (gx < 1) gx = 1;
  const dim3 grid((unsigned)gx, (unsigned)a.n_comp);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (a.f64) nodes_kernel<KIND, PREC, double><<<grid, block, 0, s>>>(P, a);
  else nodes_kernel<KIND, PREC, float><<<grid, block, 0, s>>>(P, a);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

template <int KIND, int PREC, int GRID, int NP = 1>
int launch_batch_t(const Pulse<Real<PREC>> *sets, const BatchArgs &ba, void *stream) {
  auto kern = batch_kernel<KIND, PREC, GRID, NP>;
  if constexpr (PREC == AP_FP32_PHASEFF && NP == 2 && (GRID == kGridCells || GRID == kGridCellsMix))
    kern = batch_kernel_pair_2b<KIND, GRID>;
  const int block = ba.base.shape.block;
  const size_t head = push_smem_head<PREC, GRID, NP>(block);
  const size_t smem = head + (size_t)(ba.n_sets + 1) * sizeof(long long);
  if (set_smem(kern, smem) != AP_OK) return AP_ERR_CUDA;
  int per_sm = ba.base.shape.blocks_per_sm > 0 ? ba.base.shape.blocks_per_sm
                                                : occupancy_blocks(kern, block, smem);
  const int grid = ba.base.sm_count * per_sm;
  kern<<<grid, block, smem, static_cast<cudaStream_t>(stream)>>>(sets, ba, (unsigned)head);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

// grid mode of a call: none, corners, or (float kernels) per-cell coefficients
// Whether a float-float call runs two particles per thread: requested in the
// launch shape, and a grid mode the two-particle kernels have.
inline bool pair_mode(const PushArgs &a) {
  return a.shape.pairs && (!a.grid_on || a.grid.cells);
}

template <int KIND, int PREC>
int launch_push_mode(const Pulse<Real<PREC>> &P, const PushArgs &a, void *stream) {
  if constexpr (PREC == AP_FP32_PHASEFF) {
    if (pair_mode(a))
      return !a.grid_on                 ? launch_push_pair_t<KIND, kGridNone>(P, a, stream)
             : a.shape.grid_cache == 2 ? launch_push_pair_t<KIND, kGridCellsMix>(P, a, stream)
             : a.shape.grid_cache      ? launch_push_pair_t<KIND, kGridCellsReg>(P, a, stream)
                                       : launch_push_pair_t<KIND, kGridCells>(P, a, stream);
  }
  if (!a.grid_on) return launch_push_t<KIND, PREC, kGridNone>(P, a, stream);
  if constexpr (PREC != AP_FP64) {
    if (a.grid.cells)
      return a.shape.grid_cache ? launch_push_t<KIND, PREC, kGridCellsReg>(P, a, stream)
                                : launch_push_t<KIND, PREC, kGridCells>(P, a, stream);
  }
  return launch_push_t<KIND, PREC, kGridNodes>(P, a, stream);
}

template <int KIND, int PREC>
int launch_batch_mode(const Pulse<Real<PREC>> *sets, const BatchArgs &ba, void *stream) {
  if constexpr (PREC == AP_FP32_PHASEFF) {
    if (pair_mode(ba.base))
      return !ba.base.grid_on ? launch_batch_t<KIND, PREC, kGridNone, 2>(sets, ba, stream)
             : ba.base.shape.grid_cache == 2 ? launch_batch_t<KIND, PREC, kGridCellsMix, 2>(sets, ba, stream)
             : ba.base.shape.grid_cache      ? launch_batch_t<KIND, PREC, kGridCellsReg, 2>(sets, ba, stream)
                                             : launch_batch_t<KIND, PREC, kGridCells, 2>(sets, ba, stream);
  }
  if (!ba.base.grid_on) return launch_batch_t<KIND, PREC, kGridNone>(sets, ba, stream);
  if constexpr (PREC != AP_FP64) {
    if (ba.base.grid.cells)
      return ba.base.shape.grid_cache ? launch_batch_t<KIND, PREC, kGridCellsReg>(sets, ba, stream)
                                      : launch_batch_t<KIND, PREC, kGridCells>(sets, ba, stream);
  }
  return launch_batch_t<KIND, PREC, kGridNodes>(sets, ba, stream);
}

}  // namespace apt

// Per-kind launchers: dispatch on precision and grid.
#define APT_DEFINE_KIND(K, KID)                                                                   \
  namespace apt {                                                                                 \
  int launch_push_##K(int precision, const Pulse<double> &pd, const Pulse<float> &pf,             \
                      const PushArgs &a, void *stream) {                                          \
    switch (precision) {                                                                          \
      case AP_FP64:                                                                               \
        return launch_push_mode<KID, AP_FP64>(pd, a, stream);                                     \
      case AP_FP32_PHASE64:                                                                       \
        return launch_push_mode<KID, AP_FP32_PHASE64>(pf, a, stream);                             \
      case AP_FP32_PHASEFF:                                                                       \
        return launch_push_mode<KID, AP_FP32_PHASEFF>(pf, a, stream);                             \
      default:                                                                                    \
        return AP_ERR_ARG;                                                                        \
    }                                                                                             \
  }                                                                                               \
  int launch_eval_##K(int precision, const Pulse<double> &pd, const Pulse<float> &pf,             \
                      const EvalArgs &a, void *stream) {                                          \
    switch (precision) {                                                                          \
      case AP_FP64: return launch_eval_t<KID, AP_FP64>(pd, a, stream);                            \
      case AP_FP32_PHASE64: return launch_eval_t<KID, AP_FP32_PHASE64>(pf, a, stream);            \
      case AP_FP32_PHASEFF: return launch_eval_t<KID, AP_FP32_PHASEFF>(pf, a, stream);            \
      default: return AP_ERR_ARG;                                                                 \
    }                                                                                             \
  }                                                                                               \
  int launch_nodes_##K(int precision, const Pulse<double> &pd, const Pulse<float> &pf,            \
                       const NodeArgs &a, void *stream) {                                         \
    switch (precision) {                                                                          \
      case AP_FP64: return launch_nodes_t<KID, AP_FP64>(pd, a, stream);                           \
      case AP_FP32_PHASE64: return launch_nodes_t<KID, AP_FP32_PHASE64>(pf, a, stream);           \
      case AP_FP32_PHASEFF: return launch_nodes_t<KID, AP_FP32_PHASEFF>(pf, a, stream);           \
      default: return AP_ERR_ARG;                                                                 \
    }                                                                                             \
  }                                                                                               \
  int launch_batch_##K(int precision, const Pulse<double> *dpd, const Pulse<float> *dpf,          \
                       const BatchArgs &a, void *stream) {                                        \
    switch (precision) {                                                                          \
      case AP_FP64:                                                                               \
        return launch_batch_mode<KID, AP_FP64>(dpd, a, stream);                                   \
      case AP_FP32_PHASE64:                                                                       \
        return launch_batch_mode<KID, AP_FP32_PHASE64>(dpf, a, stream);                           \
      case AP_FP32_PHASEFF:                                                                       \
        return launch_batch_mode<KID, AP_FP32_PHASEFF>(dpf, a, stream);                           \
      default:                                                                                    \
        return AP_ERR_ARG;                                                                        \
    }                                                                                             \
  }                                                                                               \
  }
