// Saxpy Map (Section 4: single-precision y = a x + y, embarrassingly parallel) and small helpers.
#include "mrw_internal.h"

namespace mrw {
namespace {

__global__ void saxpy_kernel(const float *__restrict__ x, float *__restrict__ y, int64_t n, float alpha) {
  const int64_t nv = n >> 2;
  const float4 *x4 = reinterpret_cast<const float4 *>(x);
  float4 *y4 = reinterpret_cast<float4 *>(y);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const float4 a = __ldcs(x4 + i);
    float4 b = __ldcs(y4 + i);
    b.x = fmaf(alpha, a.x, b.x);
    b.y = fmaf(alpha, a.y, b.y);
    b.z = fmaf(alpha, a.z, b.z);
    b.w = fmaf(alpha, a.w, b.w);
    __stcs(y4 + i, b);
  }
  for (int64_t i = 4 * nv + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = fmaf(alpha, x[i], y[i]);
}

__global__ void fill_u32_kernel(unsigned int *p, unsigned int v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

cudaError_t launch_saxpy(const float *x, float *y, int64_t n, float alpha, int grid, int block, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  saxpy_kernel<<<grid, block, 0, s>>>(x, y, n, alpha);
  return cudaGetLastError();
}

cudaError_t launch_fill_u32(unsigned int *p, unsigned int v, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  fill_u32_kernel<<<grid, 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

}  // namespace mrw
