// ap_grid.cu -- node-interleaved copy of the static grid field.
//
// The six component arrays of the grid (Sec. 2.1, E2/B2) are re-laid out as
// one 32-byte record per node (Ex, Ey, Ez, Bx, By, Bz, 0, 0), so that the
// refetch of a particle's cell reads 8 sectors instead of 24 (6 arrays x 4
// rows of 2 adjacent nodes).  The values are unchanged.
#include <cuda_runtime.h>

#include "ap_internal.h"

namespace {

__global__ void pack_kernel(const float *__restrict__ f0, const float *__restrict__ f1,
                            const float *__restrict__ f2, const float *__restrict__ f3,
                            const float *__restrict__ f4, const float *__restrict__ f5,
                            float4 *__restrict__ out, long long nodes) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += stride) {
    out[2 * i] = make_float4(f0[i], f1[i], f2[i], f3[i]);
    out[2 * i + 1] = make_float4(f4[i], f5[i], 0.0f, 0.0f);
  }
}

bool grid_shape_ok(const ap_grid *g) {
  return g && g->nx >= 2 && g->ny >= 2 && g->nz >= 2 &&
         (double)g->nx * g->ny * g->nz <= 2147483647.0;
}

}  // namespace

extern "C" {

size_t ap_grid_packed_bytes(const ap_grid *g) {
  if (!grid_shape_ok(g)) return 0;
  return (size_t)g->nx * g->ny * g->nz * 8 * sizeof(float);
}

int ap_grid_pack(const ap_grid *g, float *packed, void *stream) {
  if (!grid_shape_ok(g) || !packed) return AP_ERR_ARG;
  for (int c = 0; c < 6; ++c) {
    if (!g->f[c]) return AP_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(g->f[c]) & 3u) return AP_ERR_ALIGN;
  }
  if (reinterpret_cast<uintptr_t>(packed) & 15u) return AP_ERR_ALIGN;
  const long long nodes = (long long)g->nx * g->ny * g->nz;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return AP_ERR_CUDA;
  const int block = 256;
  long long want = (nodes + block - 1) / block, cap = (long long)sms * 8;
  const int grid = (int)(want < cap ? want : cap);
  pack_kernel<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(
      g->f[0], g->f[1], g->f[2], g->f[3], g->f[4], g->f[5], reinterpret_cast<float4 *>(packed), nodes);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

}  // extern "C"
