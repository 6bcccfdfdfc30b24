// ap_yee.cu -- independent 1-D vacuum Yee lines (ap_yee1d_run): the internal
// field update that the grid-node form of the technique is checked against
// (Sec. 2.1, the three-substep Yee scheme; Fig. 2e compares the analytic
// pulse with a pulse carried by this update).
//
// One block per line; the whole line (E_x on the whole nodes, B_y on the
// half nodes) stays on chip for all n_steps -- in registers, C consecutive
// nodes per thread, with only the thread-boundary values exchanged through
// shared memory (long double lines: all in shared memory) -- and is written
// back once.  Each product and difference
// is rounded separately in the stated order, so the double variant
// reproduces a plain double loop of the same expressions bit for bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "ap_internal.h"

namespace apt {
namespace {

constexpr int kYeeBlock = 1024;

__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// Register-blocked line: thread t owns the C consecutive nodes
// [t C, t C + C) of E and B in registers; per step only the two values at
// each thread boundary move, through shared memory, with two barriers:
//   (1) B half step (needs E at the next thread's first node, `en`),
//   publish the last B; barrier;
//   (2) E step (needs B at the previous thread's last node), publish the
//   first E; barrier;
//   (3) B half step with the fresh `en`.
// Each shared slot is written and read in alternate barrier intervals, so
// no write can overtake a read.  The arithmetic per node is the same as the
// plain update, so the result does not depend on C or the block size.
template <typename T, int C, int MAXT>
__global__ void __launch_bounds__(MAXT) yee1d_kernel(T *__restrict__ E, T *__restrict__ B, int nz,
                                                     T r, T hr, long long n_steps) {
  __shared__ T s_b[kYeeBlock], s_e[kYeeBlock];
  T *Eg = E + (size_t)blockIdx.x * nz;
  T *Bg = B + (size_t)blockIdx.x * nz;
  const int t = threadIdx.x;
  const int base = t * C;
  T e[C], b[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int k = base + j;
    e[j] = k < nz ? Eg[k] : T(0);
    b[j] = k < nz ? Bg[k] : T(0);
  }
  s_e[t] = e[0];
  __syncthreads();
  T en = t + 1 < (int)blockDim.x ? s_e[t + 1] : T(0);
  for (long long n = 0; n < n_steps; ++n) {
    // (1) B_{k+1/2}^{n+1/2} = B^n - (r/2)(E_{k+1}^n - E_k^n),  k <= nz - 2
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T enx = j + 1 < C ? e[j + 1] : en;
      if (base + j < nz - 1) b[j] = sub_rn(b[j], mul_rn(hr, sub_rn(enx, e[j])));
    }
    s_b[t] = b[C - 1];
    __syncthreads();
    const T bp = t > 0 ? s_b[t - 1] : T(0);
    // (2) E_k^{n+1} = E_k^n - r (B_{k+1/2}^{n+1/2} - B_{k-1/2}^{n+1/2}),  1 <= k <= nz - 1
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int k = base + j;
      const T bpv = j > 0 ? b[j - 1] : bp;
      if (k >= 1 && k < nz) e[j] = sub_rn(e[j], mul_rn(r, sub_rn(b[j], bpv)));
    }
    s_e[t] = e[0];
    __syncthreads();
    en = t + 1 < (int)blockDim.x ? s_e[t + 1] : T(0);
    // (3) B^{n+1} = B^{n+1/2} - (r/2)(E_{k+1}^{n+1} - E_k^{n+1})
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T enx = j + 1 < C ? e[j + 1] : en;
      if (base + j < nz - 1) b[j] = sub_rn(b[j], mul_rn(hr, sub_rn(enx, e[j])));
    }
  }
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int k = base + j;
    if (k < nz) {
      Eg[k] = e[j];
      Bg[k] = b[j];
    }
  }
}

template <typename T, int C, int MAXT>
int launch_yee1d_c(const ap_yee1d *y, long long n_steps, void *stream) {
  int block = ((y->nz + C - 1) / C + 31) / 32 * 32;
  if (block > MAXT) return AP_ERR_ARG;
  const double r = y->dt / y->dz;
  const double hr = 0.5 * r;
  yee1d_kernel<T, C, MAXT><<<(unsigned)y->n_lines, block, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<T *>(y->E), static_cast<T *>(y->B), y->nz, (T)r, (T)hr, n_steps);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

// Long double lines (more than 8 x 768 nodes): register arrays of that size
// would spill, so the line is kept in shared memory instead, every node
// updated by a block-stride loop with one barrier per substep (the same
// per-node arithmetic).
template <typename T>
__global__ void __launch_bounds__(kYeeBlock) yee1d_smem_kernel(T *__restrict__ E, T *__restrict__ B, int nz,
                                                               T r, T hr, long long n_steps) {
  extern __shared__ __align__(16) unsigned char yee_smem[];
  T *e = reinterpret_cast<T *>(yee_smem);
  T *b = e + nz;
  T *Eg = E + (size_t)blockIdx.x * nz;
  T *Bg = B + (size_t)blockIdx.x * nz;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    e[k] = Eg[k];
    b[k] = Bg[k];
  }
  __syncthreads();
  for (long long n = 0; n < n_steps; ++n) {
    for (int k = threadIdx.x; k < nz - 1; k += blockDim.x) b[k] = sub_rn(b[k], mul_rn(hr, sub_rn(e[k + 1], e[k])));
    __syncthreads();
    for (int k = threadIdx.x + 1; k < nz; k += blockDim.x) e[k] = sub_rn(e[k], mul_rn(r, sub_rn(b[k], b[k - 1])));
    __syncthreads();
    for (int k = threadIdx.x; k < nz - 1; k += blockDim.x) b[k] = sub_rn(b[k], mul_rn(hr, sub_rn(e[k + 1], e[k])));
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    Eg[k] = e[k];
    Bg[k] = b[k];
  }
}

template <typename T>
int launch_yee1d_smem(const ap_yee1d *y, long long n_steps, void *stream) {
  const size_t smem = 2u * sizeof(T) * (size_t)y->nz;
  auto kern = yee1d_smem_kernel<T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return AP_ERR_CUDA;
  const double r = y->dt / y->dz;
  const double hr = 0.5 * r;
  kern<<<(unsigned)y->n_lines, kYeeBlock, smem, static_cast<cudaStream_t>(stream)>>>(
      static_cast<T *>(y->E), static_cast<T *>(y->B), y->nz, (T)r, (T)hr, n_steps);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

template <typename T>
int launch_yee1d(const ap_yee1d *y, long long n_steps, void *stream) {
  const int nz = y->nz;
  // nodes per thread and block limit: the register arrays of the longer
  // lines need more than the 64 registers a 1024-thread block allows
  if (nz <= kYeeBlock) return launch_yee1d_c<T, 1, kYeeBlock>(y, n_steps, stream);
  if (nz <= 2 * kYeeBlock) return launch_yee1d_c<T, 2, kYeeBlock>(y, n_steps, stream);
  if (nz <= 4 * kYeeBlock) return launch_yee1d_c<T, 4, kYeeBlock>(y, n_steps, stream);
  if (nz <= 8 * 768) return launch_yee1d_c<T, 8, 768>(y, n_steps, stream);
  if constexpr (sizeof(T) == 8) return launch_yee1d_smem<T>(y, n_steps, stream);
  else return launch_yee1d_c<T, 16, 768>(y, n_steps, stream);
}

}  // namespace
}  // namespace apt

extern "C" int ap_yee1d_run(const ap_yee1d *y, int64_t n_steps, int32_t precision, void *stream) {
  if (!y || n_steps < 0 || y->n_lines < 0) return AP_ERR_ARG;
  if (y->nz < 2 || y->nz > AP_YEE1D_MAX_NODES) return AP_ERR_ARG;
  if (!(y->dz > 0.0) || !(y->dt > 0.0) || !(y->dz < 1e300) || !(y->dt < 1e300)) return AP_ERR_ARG;
  if (precision != AP_FP64 && precision != AP_FP32_PHASEFF) return AP_ERR_ARG;
  if (y->n_lines == 0 || n_steps == 0) return AP_OK;
  if (!y->E || !y->B) return AP_ERR_ARG;
  const uintptr_t mask = precision == AP_FP64 ? 7u : 3u;
  if (((reinterpret_cast<uintptr_t>(y->E) | reinterpret_cast<uintptr_t>(y->B)) & mask) != 0)
    return AP_ERR_ALIGN;
  return precision == AP_FP64 ? apt::launch_yee1d<double>(y, n_steps, stream)
                              : apt::launch_yee1d<float>(y, n_steps, stream);
}
