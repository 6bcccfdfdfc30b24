// ap_yee.cu -- independent 1-D vacuum Yee lines (ap_yee1d_run): the internal
// field update that the grid-node form of the technique is checked against
// (Sec. 2.1, the three-substep Yee scheme; Fig. 2e compares the analytic
// pulse with a pulse carried by this update).
//
// One block per line; the whole line (E_x on the whole nodes, B_y on the
// half nodes) stays in shared memory for all n_steps, with one barrier per
// substep, and is written back once.  Each product and difference is
// rounded separately in the stated order, so the double variant reproduces a
// plain double loop of the same expressions bit for bit.
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

template <typename T>
__global__ void __launch_bounds__(kYeeBlock) yee1d_kernel(T *__restrict__ E, T *__restrict__ B, int nz,
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
    // B_{k+1/2}^{n+1/2} = B^n - (r/2)(E_{k+1}^n - E_k^n)
    for (int k = threadIdx.x; k < nz - 1; k += blockDim.x) b[k] = sub_rn(b[k], mul_rn(hr, sub_rn(e[k + 1], e[k])));
    __syncthreads();
    // E_k^{n+1} = E_k^n - r (B_{k+1/2}^{n+1/2} - B_{k-1/2}^{n+1/2})
    for (int k = threadIdx.x + 1; k < nz; k += blockDim.x) e[k] = sub_rn(e[k], mul_rn(r, sub_rn(b[k], b[k - 1])));
    __syncthreads();
    // B^{n+1} = B^{n+1/2} - (r/2)(E_{k+1}^{n+1} - E_k^{n+1})
    for (int k = threadIdx.x; k < nz - 1; k += blockDim.x) b[k] = sub_rn(b[k], mul_rn(hr, sub_rn(e[k + 1], e[k])));
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    Eg[k] = e[k];
    Bg[k] = b[k];
  }
}

template <typename T>
int launch_yee1d(const ap_yee1d *y, long long n_steps, void *stream) {
  const size_t smem = 2u * sizeof(T) * (size_t)y->nz;
  auto kern = yee1d_kernel<T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return AP_ERR_CUDA;
  int block = ((y->nz + 31) / 32) * 32;
  if (block > kYeeBlock) block = kYeeBlock;
  const double r = y->dt / y->dz;
  const double hr = 0.5 * r;
  kern<<<(unsigned)y->n_lines, block, smem, static_cast<cudaStream_t>(stream)>>>(
      static_cast<T *>(y->E), static_cast<T *>(y->B), y->nz, (T)r, (T)hr, n_steps);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
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
