// ap_grid.cu -- packed copies of the static grid field.
//
// The six component arrays of the grid (Sec. 2.1, E2/B2) are re-laid out in
// one of two forms:
//   AP_PACK_NODES: one 32-byte record per node (Ex, Ey, Ez, Bx, By, Bz, 0, 0),
//     so that the refetch of a particle's cell reads 8 sectors instead of 24
//     (6 arrays x 4 rows of 2 adjacent nodes); the values are unchanged.
//   AP_PACK_CELLS: one 192-byte record per cell holding, per component, the
//     coefficients of the trilinear interpolant in the monomial basis
//       F(w) = a0 + a1 wx + a2 wy + a3 wz + a4 wx wy + a5 wy wz + a6 wx wz + a7 wx wy wz,
//     a0 = c000, a1 = c100 - c000, ..., a7 = the alternating sum of the 8
//     corners (cijk = corner i along x, j along y, k along z), computed in
//     double and rounded once; the refetch is one contiguous record and the
//     evaluation 7 FMA per component.  The components are interleaved in
//     pairs so that packed (f32x2) FMA evaluate two components at once.
#include <cuda_runtime.h>

#include "ap_internal.h"

namespace {

__global__ void pack_nodes_kernel(const float *__restrict__ f0, const float *__restrict__ f1,
                                  const float *__restrict__ f2, const float *__restrict__ f3,
                                  const float *__restrict__ f4, const float *__restrict__ f5,
                                  float4 *__restrict__ out, long long nodes) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += stride) {
    out[2 * i] = make_float4(f0[i], f1[i], f2[i], f3[i]);
    out[2 * i + 1] = make_float4(f4[i], f5[i], 0.0f, 0.0f);
  }
}

struct CompPtrs {
  const float *f[6];
};

// one thread per cell, x fastest; record = 12 float4 with the components
// interleaved in pairs (Ex, Ey), (Ez, Bx), (By, Bz): float 16 p + 2 k + h is
// coefficient a_k of component 2 p + h
__global__ void pack_cells_kernel(const __grid_constant__ CompPtrs src, int nx, int ny, int nz,
                                  float4 *__restrict__ out) {
  const long long cx = nx - 1, cy = ny - 1;
  const long long cells = cx * cy * (long long)(nz - 1);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long sy = nx, sz = (long long)nx * ny;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
    const long long iz = c / (cx * cy);
    const long long r = c - iz * cx * cy;
    const long long iy = r / cx;
    const long long ix = r - iy * cx;
    const long long b = iz * sz + iy * sy + ix;
    float *rec = reinterpret_cast<float *>(out + 12 * c);
    for (int comp = 0; comp < 6; ++comp) {
      const float *f = src.f[comp];
      const double c000 = f[b], c100 = f[b + 1], c010 = f[b + sy], c110 = f[b + sy + 1];
      const double c001 = f[b + sz], c101 = f[b + sz + 1], c011 = f[b + sz + sy],
                   c111 = f[b + sz + sy + 1];
      const double a1 = c100 - c000, a2 = c010 - c000, a3 = c001 - c000;
      const double a4 = (c110 - c100) - (c010 - c000);
      const double a5 = (c011 - c010) - (c001 - c000);
      const double a6 = (c101 - c100) - (c001 - c000);
      const double a7 = ((c111 - c110) - (c101 - c100)) - ((c011 - c010) - (c001 - c000));
      const double a[8] = {c000, a1, a2, a3, a4, a5, a6, a7};
      float *r = rec + 16 * (comp >> 1) + (comp & 1);
      for (int k = 0; k < 8; ++k) r[2 * k] = (float)a[k];
    }
  }
}

bool grid_shape_ok(const ap_grid *g) {
  return g && g->nx >= 2 && g->ny >= 2 && g->nz >= 2 &&
         (double)g->nx * g->ny * g->nz <= 2147483647.0 &&
         (g->packed_layout == AP_PACK_NODES || g->packed_layout == AP_PACK_CELLS);
}

}  // namespace

extern "C" {

size_t ap_grid_packed_bytes(const ap_grid *g) {
  if (!grid_shape_ok(g)) return 0;
  if (g->packed_layout == AP_PACK_CELLS)
    return (size_t)(g->nx - 1) * (g->ny - 1) * (g->nz - 1) * 48 * sizeof(float);
  return (size_t)g->nx * g->ny * g->nz * 8 * sizeof(float);
}

int ap_grid_pack(const ap_grid *g, float *packed, void *stream) {
  if (!grid_shape_ok(g) || !packed) return AP_ERR_ARG;
  for (int c = 0; c < 6; ++c) {
    if (!g->f[c]) return AP_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(g->f[c]) & 3u) return AP_ERR_ALIGN;
  }
  if (reinterpret_cast<uintptr_t>(packed) & 15u) return AP_ERR_ALIGN;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return AP_ERR_CUDA;
  const int block = 256;
  const long long cap = (long long)sms * 8;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->packed_layout == AP_PACK_CELLS) {
    const long long cells = (long long)(g->nx - 1) * (g->ny - 1) * (g->nz - 1);
    const long long want = (cells + block - 1) / block;
    CompPtrs src;
    for (int c = 0; c < 6; ++c) src.f[c] = g->f[c];
    pack_cells_kernel<<<(int)(want < cap ? want : cap), block, 0, s>>>(src, g->nx, g->ny, g->nz,
                                                                      reinterpret_cast<float4 *>(packed));
  } else {
    const long long nodes = (long long)g->nx * g->ny * g->nz;
    const long long want = (nodes + block - 1) / block;
    pack_nodes_kernel<<<(int)(want < cap ? want : cap), block, 0, s>>>(
        g->f[0], g->f[1], g->f[2], g->f[3], g->f[4], g->f[5], reinterpret_cast<float4 *>(packed), nodes);
  }
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

}  // extern "C"
