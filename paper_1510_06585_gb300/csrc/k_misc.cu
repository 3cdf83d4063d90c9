// Saxpy Map (Section 4: single-precision y = a x + y, embarrassingly parallel) and small helpers.
#include <algorithm>

#include "mrw_internal.h"

namespace mrw {
namespace {

// A Map of k saxpy stages over the same x (Section 4, Saxpy): y := alpha_s x + y for s = 0 .. k-1,
// in order, in registers, one fused multiply-add per stage and element, so the result has the bits
// of k single-stage launches. One HBM read of x and of y and one write of y per element.
// CTA b owns the float4 groups [b * 256 * U, (b + 1) * 256 * U), thread t the groups t, t + 256, ...
// of it: each thread issues its 2U 16-byte loads before any arithmetic (U loads of x and of y in
// flight), and the grid has one CTA per tile, scheduled as SMs free up.
template <int U>
__global__ void __launch_bounds__(256) saxpy_kernel(const __grid_constant__ SaxpyArgs a) {
  const int64_t nv = a.n >> 2;
  const float4 *x4 = reinterpret_cast<const float4 *>(a.x);
  float4 *y4 = reinterpret_cast<float4 *>(a.y);
  const int64_t base = (int64_t)blockIdx.x * (256 * U) + threadIdx.x;
  float4 xv[U], yv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = base + (int64_t)u * 256;
    if (i < nv) {
      xv[u] = __ldcs(x4 + i);
      yv[u] = __ldcs(y4 + i);
    }
  }
  for (int s = 0; s < a.nstages; ++s) {
    const float al = a.alpha[s];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      yv[u].x = fmaf(al, xv[u].x, yv[u].x);
      yv[u].y = fmaf(al, xv[u].y, yv[u].y);
      yv[u].z = fmaf(al, xv[u].z, yv[u].z);
      yv[u].w = fmaf(al, xv[u].w, yv[u].w);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = base + (int64_t)u * 256;
    if (i < nv) __stcs(y4 + i, yv[u]);
  }
  // the n mod 4 trailing elements: the first threads of the last CTA
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x < (a.n & 3)) {
    const int64_t i = 4 * nv + threadIdx.x;
    float yi = a.y[i];
    const float xi = a.x[i];
    for (int s = 0; s < a.nstages; ++s) yi = fmaf(a.alpha[s], xi, yi);
    a.y[i] = yi;
  }
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

cudaError_t compare_copy_node(const uint8_t *b, uint8_t *a, int64_t rows, int32_t W, int64_t pitch,
                              unsigned int *changed, int sms, NodeChain &nc) {
  const int64_t n = rows * ((W + 15) / 16);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  void *args[] = {(void *)&b, (void *)&a, (void *)&rows, (void *)&W, (void *)&pitch, (void *)&changed};
  return nc.kernel((const void *)compare_copy_kernel, dim3(grid > 0 ? grid : 1), dim3(256), 0, args);
}

cudaError_t while_control_node(LoopCtrl *ctrl, unsigned int *changed, cudaGraphConditionalHandle h, NodeChain &nc) {
  void *args[] = {(void *)&ctrl, (void *)&changed, (void *)&h};
  return nc.kernel((const void *)while_control_kernel, dim3(1), dim3(1), 0, args);
}

cudaError_t while_init_node(LoopCtrl *ctrl, unsigned int *words, unsigned long long max_iters, NodeChain &nc) {
  void *args[] = {(void *)&ctrl, (void *)&words, (void *)&max_iters};
  return nc.kernel((const void *)while_init_kernel, dim3(1), dim3(1), 0, args);
}

int saxpy_grid(int64_t n, int unroll) {
  const int64_t tiles = ((n >> 2) + 256LL * unroll - 1) / (256LL * unroll);
  return (int)std::max<int64_t>(1, tiles);
}

cudaError_t launch_saxpy(const SaxpyArgs &a, int unroll, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (a.nstages < 1 || a.nstages > kMaxSaxpyStages) return cudaErrorInvalidValue;
  const int64_t tiles = ((a.n >> 2) + 256LL * unroll - 1) / (256LL * unroll);
  if (tiles > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  const int grid = saxpy_grid(a.n, unroll);
  switch (unroll) {
    case 1: saxpy_kernel<1><<<grid, 256, 0, s>>>(a); break;
    case 2: saxpy_kernel<2><<<grid, 256, 0, s>>>(a); break;
    case 4: saxpy_kernel<4><<<grid, 256, 0, s>>>(a); break;
    case 8: saxpy_kernel<8><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mrw
