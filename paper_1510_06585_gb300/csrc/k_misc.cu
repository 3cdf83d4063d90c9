// Saxpy Map (Section 4: single-precision y = a x + y, embarrassingly parallel) and small helpers.
#include <algorithm>

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

// a := b where they differ (rows of W bytes, both with `pitch`, 16-byte aligned rows) and
// *changed := 1 if any byte differed.
__global__ void compare_copy_kernel(const uint8_t *__restrict__ b, uint8_t *__restrict__ a, int64_t rows, int32_t W,
                                    int64_t pitch, unsigned int *changed) {
  const int col_vecs = (W + 15) >> 4;
  const int64_t n = rows * col_vecs;
  bool diff = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / col_vecs;
    const int c = (int)(i - r * col_vecs) * 16;
    const uint8_t *pb = b + r * pitch + c;
    uint8_t *pa = a + r * pitch + c;
    if (c + 16 <= W) {
      const uint4 vb = *reinterpret_cast<const uint4 *>(pb);
      const uint4 va = *reinterpret_cast<const uint4 *>(pa);
      if (vb.x != va.x || vb.y != va.y || vb.z != va.z || vb.w != va.w) {
        *reinterpret_cast<uint4 *>(pa) = vb;
        diff = true;
      }
    } else {
      for (int k = 0; c + k < W; ++k)
        if (pa[k] != pb[k]) {
          pa[k] = pb[k];
          diff = true;
        }
    }
  }
  if (__any_sync(0xFFFFFFFFu, diff) && (threadIdx.x & 31) == 0) *changed = 1u;
}

// One run of a WHILE_CHANGED loop body has finished: count it and continue while it changed its
// input and the iteration bound is not reached; clear the flag for the next run.
__global__ void while_control_kernel(LoopCtrl *ctrl, unsigned int *changed, cudaGraphConditionalHandle h) {
  const unsigned long long it = ctrl->iter + 1;
  ctrl->iter = it;
  const unsigned int c = *changed;
  *changed = 0u;
  cudaGraphSetConditional(h, (c != 0u && it < ctrl->max_iters) ? 1u : 0u);
}

// words[0] = changed flag, words[1] = status word of the loop body's stencil launches
__global__ void while_init_kernel(LoopCtrl *ctrl, unsigned int *words, unsigned long long max_iters) {
  ctrl->iter = 0;
  ctrl->max_iters = max_iters;
  words[0] = 0u;
  words[1] = 0u;
}

}  // namespace

cudaError_t launch_compare_copy(const uint8_t *b, uint8_t *a, int64_t rows, int32_t W, int64_t pitch,
                                unsigned int *changed, int sms, cudaStream_t s) {
  const int64_t n = rows * ((W + 15) / 16);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  compare_copy_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(b, a, rows, W, pitch, changed);
  return cudaGetLastError();
}

cudaError_t launch_while_control(LoopCtrl *ctrl, unsigned int *changed, cudaGraphConditionalHandle h, cudaStream_t s) {
  while_control_kernel<<<1, 1, 0, s>>>(ctrl, changed, h);
  return cudaGetLastError();
}

cudaError_t launch_while_init(LoopCtrl *ctrl, unsigned int *changed, unsigned long long max_iters, cudaStream_t s) {
  while_init_kernel<<<1, 1, 0, s>>>(ctrl, changed, max_iters);
  return cudaGetLastError();
}

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
