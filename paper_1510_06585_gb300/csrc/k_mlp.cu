// Cost-model MLP kernels: 16 -> H -> H -> K, ReLU, bf16 weights, fp32 accumulation.
//
// The paper derives configurations for unseen (SCT, workload) pairs by interpolating stored
// profiles (Section 3.2, Configuration Derivation). The executor learns that mapping instead; the
// network is small (a few thousand weights), so the kernels favour latency: each CTA stages the
// bf16 weights once as fp32 in shared memory and processes a chunk of samples whose activations
// also stay in shared memory. The backward pass turns the chunk's per-sample deltas into weight
// gradients as small matrix products over the chunk and adds them to the global gradient with one
// atomic per weight per CTA. No tensor cores: the contractions are 16..128 wide.
#include <cuda_bf16.h>

#include "mrw_internal.h"

namespace mrw {
namespace {

constexpr int kBlock = 256;
constexpr int kChunk = 32;  // samples per CTA pass

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

struct Smem {
  float *w1, *b1, *w2, *b2, *w3, *b3;
  float *x, *z1, *z2, *y, *d2, *d1;
};

__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ Smem carve(float *base, const MlpDims &d) {
  Smem s;
  const int H = d.hidden, K = d.k, I = d.nin;
  s.w1 = base;
  s.b1 = s.w1 + H * I;
  s.w2 = s.b1 + H;
  s.b2 = s.w2 + H * H;
  s.w3 = s.b2 + H;
  s.b3 = s.w3 + K * H;
  s.x = s.b3 + K;
  s.z1 = s.x + kChunk * I;
  s.z2 = s.z1 + kChunk * H;
  s.y = s.z2 + kChunk * H;
  s.d2 = s.y + kChunk * K;
  s.d1 = s.d2 + kChunk * H;
  return s;
}

__device__ void load_weights(const Smem &s, const MlpDims &d, const uint16_t *wbf) {
  for (int64_t i = threadIdx.x; i < d.nparams; i += blockDim.x) s.w1[i] = bf2f(wbf[i]);
}

// Forward over `cnt` samples already in s.x: fills z1, z2 (pre-activations) and y.
__device__ void forward_chunk(const Smem &s, const MlpDims &d, int cnt) {
  const int H = d.hidden, K = d.k, I = d.nin;
  for (int e = threadIdx.x; e < cnt * H; e += blockDim.x) {
    const int n = e / H, o = e % H;
    float acc = s.b1[o];
    for (int i = 0; i < I; ++i) acc = fmaf(s.w1[o * I + i], s.x[n * I + i], acc);
    s.z1[n * H + o] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < cnt * H; e += blockDim.x) {
    const int n = e / H, o = e % H;
    float acc = s.b2[o];
    for (int i = 0; i < H; ++i) acc = fmaf(s.w2[o * H + i], fmaxf(s.z1[n * H + i], 0.f), acc);
    s.z2[n * H + o] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < cnt * K; e += blockDim.x) {
    const int n = e / K, o = e % K;
    float acc = s.b3[o];
    for (int i = 0; i < H; ++i) acc = fmaf(s.w3[o * H + i], fmaxf(s.z2[n * H + i], 0.f), acc);
    s.y[n * K + o] = acc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBlock) forward_kernel(MlpDims d, const uint16_t *__restrict__ wbf,
                                                         const float *__restrict__ x, int64_t n,
                                                         float *__restrict__ y) {
  extern __shared__ float sm[];
  const Smem s = carve(sm, d);
  load_weights(s, d, wbf);
  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < n; c0 += (int64_t)gridDim.x * kChunk) {
    const int cnt = (int)imin64(kChunk, n - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * d.nin; e += blockDim.x) s.x[e] = x[c0 * d.nin + e];
    __syncthreads();
    forward_chunk(s, d, cnt);
    for (int e = threadIdx.x; e < cnt * d.k; e += blockDim.x) y[c0 * d.k + e] = s.y[e];
  }
}

__global__ void __launch_bounds__(kBlock) backward_kernel(MlpDims d, const uint16_t *__restrict__ wbf,
                                                          const float *__restrict__ x, const float *__restrict__ t,
                                                          const int32_t *__restrict__ idx, int64_t n, float scale,
                                                          float *__restrict__ g, float *__restrict__ loss_acc) {
  extern __shared__ float sm[];
  const Smem s = carve(sm, d);
  const int H = d.hidden, K = d.k, I = d.nin;
  load_weights(s, d, wbf);
  __shared__ float s_loss[kBlock / 32];
  float my_loss = 0.f;
  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < n; c0 += (int64_t)gridDim.x * kChunk) {
    const int cnt = (int)imin64(kChunk, n - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * I; e += blockDim.x) {
      const int r = e / I, c = e % I;
      const int64_t src = idx ? idx[c0 + r] : c0 + r;
      s.x[e] = x[src * I + c];
    }
    __syncthreads();
    forward_chunk(s, d, cnt);
    // dL/dy = 2 (y - t) * scale, scale = 1 / (batch * K)
    for (int e = threadIdx.x; e < cnt * K; e += blockDim.x) {
      const int r = e / K, c = e % K;
      const int64_t src = idx ? idx[c0 + r] : c0 + r;
      const float diff = s.y[e] - t[src * K + c];
      my_loss = fmaf(diff, diff, my_loss);
      s.y[e] = 2.f * diff * scale;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * H; e += blockDim.x) {
      const int r = e / H, i = e % H;
      float acc = 0.f;
      for (int k = 0; k < K; ++k) acc = fmaf(s.w3[k * H + i], s.y[r * K + k], acc);
      s.d2[e] = s.z2[e] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * H; e += blockDim.x) {
      const int r = e / H, i = e % H;
      float acc = 0.f;
      for (int o = 0; o < H; ++o) acc = fmaf(s.w2[o * H + i], s.d2[r * H + o], acc);
      s.d1[e] = s.z1[e] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // weight gradients over the chunk
    float *gw1 = g + d.off_w1, *gb1 = g + d.off_b1, *gw2 = g + d.off_w2, *gb2 = g + d.off_b2;
    float *gw3 = g + d.off_w3, *gb3 = g + d.off_b3;
    for (int e = threadIdx.x; e < K * H; e += blockDim.x) {
      const int k = e / H, i = e % H;
      float acc = 0.f;
      for (int r = 0; r < cnt; ++r) acc = fmaf(s.y[r * K + k], fmaxf(s.z2[r * H + i], 0.f), acc);
      atomicAdd(gw3 + e, acc);
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < cnt; ++r) acc += s.y[r * K + k];
      atomicAdd(gb3 + k, acc);
    }
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
      const int o = e / H, i = e % H;
      float acc = 0.f;
      for (int r = 0; r < cnt; ++r) acc = fmaf(s.d2[r * H + o], fmaxf(s.z1[r * H + i], 0.f), acc);
      atomicAdd(gw2 + e, acc);
    }
    for (int o = threadIdx.x; o < H; o += blockDim.x) {
      float a2 = 0.f, a1 = 0.f;
      for (int r = 0; r < cnt; ++r) {
        a2 += s.d2[r * H + o];
        a1 += s.d1[r * H + o];
      }
      atomicAdd(gb2 + o, a2);
      atomicAdd(gb1 + o, a1);
    }
    for (int e = threadIdx.x; e < H * I; e += blockDim.x) {
      const int o = e / I, i = e % I;
      float acc = 0.f;
      for (int r = 0; r < cnt; ++r) acc = fmaf(s.d1[r * H + o], s.x[r * I + i], acc);
      atomicAdd(gw1 + e, acc);
    }
  }
  // block-reduce the squared errors
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xFFFFFFFFu, my_loss, o);
  if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = my_loss;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f;
    for (int i = 0; i < kBlock / 32; ++i) tot += s_loss[i];
    atomicAdd(loss_acc, tot);
  }
}

__global__ void round_kernel(const float *__restrict__ m, uint16_t *__restrict__ bf, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bf[i] = __bfloat16_as_ushort(__float2bfloat16_rn(m[i]));
}

__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                            float bc1, float bc2, uint16_t *__restrict__ bf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    bf[i] = __bfloat16_as_ushort(__float2bfloat16_rn(wi));
  }
}

size_t smem_bytes(const MlpDims &d) {
  const int64_t act = (int64_t)kChunk * (d.nin + 4 * d.hidden + d.k);
  return (size_t)(d.nparams + act) * sizeof(float);
}

bool smem_attr(const void *fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

}  // namespace

MlpDims mlp_dims(int nin, int hidden, int k) {
  MlpDims d;
  d.nin = nin;
  d.hidden = hidden;
  d.k = k;
  d.off_w1 = 0;
  d.off_b1 = d.off_w1 + (int64_t)hidden * nin;
  d.off_w2 = d.off_b1 + hidden;
  d.off_b2 = d.off_w2 + (int64_t)hidden * hidden;
  d.off_w3 = d.off_b2 + hidden;
  d.off_b3 = d.off_w3 + (int64_t)k * hidden;
  d.nparams = d.off_b3 + k;
  return d;
}

cudaError_t launch_mlp_round_bf16(const float *master, uint16_t *bf, int64_t n, cudaStream_t s) {
  round_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(master, bf, n);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const MlpDims &d, const uint16_t *wbf, const float *x, int64_t n, float *y,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sb = smem_bytes(d);
  if (!smem_attr((const void *)forward_kernel, sb)) return cudaErrorInvalidValue;
  const int grid = (int)imin64((n + kChunk - 1) / kChunk, 304);
  forward_kernel<<<grid, kBlock, sb, s>>>(d, wbf, x, n, y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const MlpDims &d, const uint16_t *wbf, const float *x, const float *t,
                                const int32_t *idx, int64_t n, float scale, float *grads, float *loss_acc,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t sb = smem_bytes(d);
  if (!smem_attr((const void *)backward_kernel, sb)) return cudaErrorInvalidValue;
  const int grid = (int)imin64((n + kChunk - 1) / kChunk, 152);
  backward_kernel<<<grid, kBlock, sb, s>>>(d, wbf, x, t, idx, n, scale, grads, loss_acc);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *master, float *m, float *v, const float *g, int64_t n, float lr, float b1,
                            float b2, float eps, float bc1, float bc2, uint16_t *bf, cudaStream_t s) {
  adam_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(master, m, v, g, n, lr, b1, b2, eps, bc1, bc2, bf);
  return cudaGetLastError();
}

}  // namespace mrw
