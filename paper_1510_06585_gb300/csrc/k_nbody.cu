// N-body on the Loop skeleton (Section 4, N-Body): direct-sum forces with the positions given
// whole to every partition (COPY transfer mode, Section 3.4) and a synchronisation between
// iterations; kick-drift-kick leapfrog.
//
// Partitioning: the bodies are split into one contiguous range per CTA (the paper's partitions,
// here one per SM-resident CTA); each thread owns `B` bodies of its CTA's range, strided by the
// block size so that loads and stores stay coalesced. Every CTA streams all positions through a
// shared-memory tile (the COPY vector) and sums j in index order, so each body's sum has the same
// order whatever the launch shape — Loop(k) and k single steps give bit-identical states.
//
// Loop (Section 2.1; the paper evaluates the condition on the host, Section 3.1): here the
// condition is evaluated on the device. One step is two kernels (drift, then force + kick):
// the launch boundary is the global synchronisation. The steps run inside a CUDA graph whose
// conditional WHILE node re-runs its body while the device-side counter is below max_iters; the
// drift kernel's first thread advances the counter and sets the condition.
#include "mrw_internal.h"

namespace mrw {
namespace {

constexpr int kTile = 256;

template <int B>
__global__ void __launch_bounds__(256) force_kernel(const float4 *__restrict__ x, float4 *__restrict__ v,
                                                    float4 *__restrict__ a, int n, float G, float eps2, float hdt,
                                                    int kick) {
  __shared__ float4 tile[kTile];
  const int64_t lo = (int64_t)n * blockIdx.x / gridDim.x;
  const int64_t hi = (int64_t)n * (blockIdx.x + 1) / gridDim.x;
  float3 xi[B];
  float3 acc[B];
  int idx[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int64_t i = lo + threadIdx.x + (int64_t)b * blockDim.x;
    idx[b] = i < hi ? (int)i : -1;
    const float4 p = idx[b] >= 0 ? x[idx[b]] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[b] = make_float3(p.x, p.y, p.z);
    acc[b] = make_float3(0.f, 0.f, 0.f);
  }
  for (int j0 = 0; j0 < n; j0 += kTile) {
    __syncthreads();
    for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
      // zero-mass padding adds exactly zero to every sum
      tile[k] = j0 + k < n ? x[j0 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kTile; ++k) {
      const float4 pj = tile[k];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const float dx = pj.x - xi[b].x;
        const float dy = pj.y - xi[b].y;
        const float dz = pj.z - xi[b].z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        const float inv = rsqrtf(r2);
        const float s = (pj.w * inv) * (inv * inv);
        acc[b].x = fmaf(s, dx, acc[b].x);
        acc[b].y = fmaf(s, dy, acc[b].y);
        acc[b].z = fmaf(s, dz, acc[b].z);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if (idx[b] < 0) continue;
    const float4 ai = make_float4(G * acc[b].x, G * acc[b].y, G * acc[b].z, 0.f);
    a[idx[b]] = ai;
    if (kick) {
      float4 vi = v[idx[b]];
      vi.x = fmaf(hdt, ai.x, vi.x);
      vi.y = fmaf(hdt, ai.y, vi.y);
      vi.z = fmaf(hdt, ai.z, vi.z);
      v[idx[b]] = vi;
    }
  }
}

// v += dt/2 a; x += dt v. With ctrl != nullptr the first thread also advances the Loop counter
// and sets the graph condition for the next iteration.
__global__ void drift_kernel(float4 *__restrict__ x, float4 *__restrict__ v, const float4 *__restrict__ a, int n,
                             float dt, LoopCtrl *ctrl, cudaGraphConditionalHandle h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (ctrl != nullptr && i == 0) {
    const unsigned long long it = ctrl->iter + 1;
    ctrl->iter = it;
    cudaGraphSetConditional(h, it < ctrl->max_iters ? 1u : 0u);
  }
  if (i < n) {
    const float hdt = 0.5f * dt;
    float4 vi = v[i];
    const float4 ai = a[i];
    float4 xi = x[i];
    vi.x = fmaf(hdt, ai.x, vi.x);
    vi.y = fmaf(hdt, ai.y, vi.y);
    vi.z = fmaf(hdt, ai.z, vi.z);
    xi.x = fmaf(dt, vi.x, xi.x);
    xi.y = fmaf(dt, vi.y, xi.y);
    xi.z = fmaf(dt, vi.z, xi.z);
    v[i] = vi;
    x[i] = xi;
  }
}

__global__ void kick_kernel(float4 *__restrict__ v, const float4 *__restrict__ a, int n, float hdt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float4 vi = v[i];
    const float4 ai = a[i];
    vi.x = fmaf(hdt, ai.x, vi.x);
    vi.y = fmaf(hdt, ai.y, vi.y);
    vi.z = fmaf(hdt, ai.z, vi.z);
    v[i] = vi;
  }
}

__global__ void loop_init_kernel(LoopCtrl *ctrl, unsigned long long max_iters) {
  ctrl->iter = 0;
  ctrl->max_iters = max_iters;
}

void *force_fn(int b) {
  switch (b) {
    case 1: return (void *)force_kernel<1>;
    case 4: return (void *)force_kernel<4>;
    default: return (void *)force_kernel<2>;
  }
}

}  // namespace

cudaError_t launch_nbody_force(const NBodyParams &p, int kick, int bpt, int grid, int block, cudaStream_t s) {
  const float hdt = 0.5f * p.dt;
  switch (bpt) {
    case 1: force_kernel<1><<<grid, block, 0, s>>>(p.x, p.v, p.a, p.n, p.G, p.eps2, hdt, kick); break;
    case 4: force_kernel<4><<<grid, block, 0, s>>>(p.x, p.v, p.a, p.n, p.G, p.eps2, hdt, kick); break;
    default: force_kernel<2><<<grid, block, 0, s>>>(p.x, p.v, p.a, p.n, p.G, p.eps2, hdt, kick); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_nbody_drift(const NBodyParams &p, cudaStream_t s) {
  const int block = 256, grid = (p.n + block - 1) / block;
  drift_kernel<<<grid, block, 0, s>>>(p.x, p.v, p.a, p.n, p.dt, nullptr, cudaGraphConditionalHandle{});
  return cudaGetLastError();
}

cudaError_t launch_nbody_kick(const NBodyParams &p, cudaStream_t s) {
  const int block = 256, grid = (p.n + block - 1) / block;
  kick_kernel<<<grid, block, 0, s>>>(p.v, p.a, p.n, 0.5f * p.dt);
  return cudaGetLastError();
}

#define MRW_TRY(call)                       \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) {                \
      if (graph) cudaGraphDestroy(graph);   \
      return e_;                            \
    }                                       \
  } while (0)

cudaError_t build_nbody_loop_graph(const NBodyParams &p, LoopCtrl *ctrl, int64_t iters, int bpt, int grid,
                                   int block, cudaGraphExec_t *exec) {
  cudaGraph_t graph = nullptr;
  MRW_TRY(cudaGraphCreate(&graph, 0));

  // node 1: reset the counter
  cudaGraphNode_t init_node;
  {
    unsigned long long mi = (unsigned long long)iters;
    void *args[] = {(void *)&ctrl, (void *)&mi};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)loop_init_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    MRW_TRY(cudaGraphAddKernelNode(&init_node, graph, nullptr, 0, &kp));
  }

  // node 2: WHILE (condition) { body } with the condition 1 at entry when iters > 0
  cudaGraphConditionalHandle handle;
  MRW_TRY(cudaGraphConditionalHandleCreate(&handle, graph, iters > 0 ? 1u : 0u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cparams = {};
  cparams.type = cudaGraphNodeTypeConditional;
  cparams.conditional.handle = handle;
  cparams.conditional.type = cudaGraphCondTypeWhile;
  cparams.conditional.size = 1;
  cudaGraphNode_t cond_node;
  MRW_TRY(cudaGraphAddNode(&cond_node, graph, &init_node, nullptr, 1, &cparams));
  cudaGraph_t body = cparams.conditional.phGraph_out[0];

  // body: drift (advances the counter, sets the condition) -> force + kick
  cudaGraphNode_t drift_node, force_node;
  {
    float4 *xx = p.x, *vv = p.v, *aa = p.a;
    int n = p.n;
    float dt = p.dt;
    LoopCtrl *c = ctrl;
    cudaGraphConditionalHandle h = handle;
    void *args[] = {(void *)&xx, (void *)&vv, (void *)&aa, (void *)&n, (void *)&dt, (void *)&c, (void *)&h};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)drift_kernel;
    kp.gridDim = dim3((p.n + 255) / 256);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    MRW_TRY(cudaGraphAddKernelNode(&drift_node, body, nullptr, 0, &kp));
  }
  {
    const float4 *xx = p.x;
    float4 *vv = p.v, *aa = p.a;
    int n = p.n;
    float G = p.G, eps2 = p.eps2, hdt = 0.5f * p.dt;
    int kick = 1;
    void *args[] = {(void *)&xx, (void *)&vv, (void *)&aa, (void *)&n, (void *)&G, (void *)&eps2, (void *)&hdt,
                    (void *)&kick};
    cudaKernelNodeParams kp = {};
    kp.func = force_fn(bpt);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.kernelParams = args;
    MRW_TRY(cudaGraphAddKernelNode(&force_node, body, &drift_node, 1, &kp));
  }
  cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

}  // namespace mrw
