// N-body on the Loop skeleton (Section 4, N-Body): direct-sum forces with the positions given
// whole to every partition (COPY transfer mode, Section 3.4) and a synchronisation between
// iterations; kick-drift-kick leapfrog.
//
// Partitioning: the bodies are split into one contiguous range per CTA (the paper's partitions,
// here one per SM-resident CTA); each thread owns `B` bodies of its CTA's range, strided by the
// group size so that loads and stores stay coalesced. A CTA has four warp groups; each streams a
// fixed quarter of all positions (the COPY vector) through its own shared-memory tile, so an SM
// runs four times as many warps as 65536 bodies alone would give it. Arithmetic uses the packed
// f32x2 instructions of sm_100+: the two lanes of a register pair hold an even j and the next odd
// j, halving the instruction count per interaction. Each body's sum has a fixed order that depends
// on N only (pairs in index order per lane, lanes added, quarters added in order), so Loop(k) and k
// single steps, and every launch shape, give bit-identical states.
//
// Loop (Section 2.1; the paper evaluates the condition on the host, Section 3.1): here the
// condition is evaluated on the device. One step is two kernels (drift, then force + kick):
// the launch boundary is the global synchronisation. The steps run inside a CUDA graph whose
// conditional WHILE node re-runs its body while the device-side counter is below max_iters; the
// drift kernel's first thread advances the counter and sets the condition.
#include "mrw_internal.h"

namespace mrw {
namespace {

constexpr int kJSplit = 4;   // warp groups per CTA, each summing a fixed quarter of the j range
constexpr int kTileJ = 256;  // j bodies per shared-memory tile and group

// Packed FP32 pairs (sm_100+ f32x2 instructions): lane 0 holds an even j, lane 1 the next odd j.
__device__ __forceinline__ unsigned long long pk(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void group_sync(int g, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(nthreads) : "memory");
}

// First j of group g (even, so pairs never straddle two groups); group kJSplit ends at n.
__device__ __forceinline__ int group_start(int n, int g) {
  return g >= kJSplit ? n : (int)(((int64_t)n * g / kJSplit) & ~1LL);
}

// Accelerations of the CTA's bodies [lo, hi) with hi - lo <= T * B, T = blockDim.x / kJSplit.
// Every body's sum: per group, pairs (j, j+1) accumulated lane-wise in index order, lanes added;
// then the groups' partial sums added in group order. The order depends on n only.
template <int B>
__global__ void __launch_bounds__(B == 4 ? 512 : 1024, 1) force_kernel(const float4 *__restrict__ x, float4 *__restrict__ v,
                                                        float4 *__restrict__ a, int n, float G, float eps2,
                                                        float hdt, int kick) {
  __shared__ __align__(16) float tile[kJSplit][4][kTileJ];
  extern __shared__ float part[];  // [kJSplit][3][T * B]
  const int T = blockDim.x / kJSplit;
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const int64_t lo = (int64_t)n * blockIdx.x / gridDim.x;
  const int64_t hi = (int64_t)n * (blockIdx.x + 1) / gridDim.x;

  unsigned long long xi[B], yi[B], zi[B], ax[B], ay[B], az[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int64_t i = lo + t + (int64_t)b * T;
    const float4 p = i < hi ? x[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[b] = pk(p.x, p.x);
    yi[b] = pk(p.y, p.y);
    zi[b] = pk(p.z, p.z);
    ax[b] = ay[b] = az[b] = 0ull;
  }
  const unsigned long long e2 = pk(eps2, eps2);
  const int j_begin = group_start(n, g), j_end = group_start(n, g + 1);
  float *tx = tile[g][0], *ty = tile[g][1], *tz = tile[g][2], *tm = tile[g][3];
  for (int j0 = j_begin; j0 < j_end; j0 += kTileJ) {
    group_sync(g, T);
    for (int k = t; k < kTileJ; k += T) {
      // zero-mass padding adds exactly zero to every sum
      const float4 q = j0 + k < j_end ? x[j0 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
      tx[k] = q.x;
      ty[k] = q.y;
      tz[k] = q.z;
      tm[k] = q.w;
    }
    group_sync(g, T);
    const int kend = min(kTileJ, j_end - j0 + 1) & ~1;  // pairs covering the valid j of this tile
#pragma unroll 4
    for (int k = 0; k < kend; k += 2) {
      const unsigned long long x2 = *reinterpret_cast<const unsigned long long *>(tx + k);
      const unsigned long long y2 = *reinterpret_cast<const unsigned long long *>(ty + k);
      const unsigned long long z2 = *reinterpret_cast<const unsigned long long *>(tz + k);
      const unsigned long long m2 = *reinterpret_cast<const unsigned long long *>(tm + k);
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const unsigned long long dx = sub2(x2, xi[b]);
        const unsigned long long dy = sub2(y2, yi[b]);
        const unsigned long long dz = sub2(z2, zi[b]);
        const unsigned long long r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e2)));
        const float2 rr = upk(r2);
        const unsigned long long inv = pk(rsqrt_approx(rr.x), rsqrt_approx(rr.y));
        const unsigned long long s = mul2(mul2(m2, inv), mul2(inv, inv));
        ax[b] = fma2(s, dx, ax[b]);
        ay[b] = fma2(s, dy, ay[b]);
        az[b] = fma2(s, dz, az[b]);
      }
    }
  }
  const int nb = T * B;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const float2 px = upk(ax[b]), py = upk(ay[b]), pz = upk(az[b]);
    const int li = t + b * T;
    part[(g * 3 + 0) * nb + li] = px.x + px.y;
    part[(g * 3 + 1) * nb + li] = py.x + py.y;
    part[(g * 3 + 2) * nb + li] = pz.x + pz.y;
  }
  __syncthreads();
  if (g != 0) return;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int li = t + b * T;
    const int64_t i = lo + li;
    if (i >= hi) continue;
    float sx = part[0 * nb + li], sy = part[1 * nb + li], sz = part[2 * nb + li];
#pragma unroll
    for (int q = 1; q < kJSplit; ++q) {
      sx += part[(q * 3 + 0) * nb + li];
      sy += part[(q * 3 + 1) * nb + li];
      sz += part[(q * 3 + 2) * nb + li];
    }
    const float4 ai = make_float4(G * sx, G * sy, G * sz, 0.f);
    a[i] = ai;
    if (kick) {
      float4 vi = v[i];
      vi.x = fmaf(hdt, ai.x, vi.x);
      vi.y = fmaf(hdt, ai.y, vi.y);
      vi.z = fmaf(hdt, ai.z, vi.z);
      v[i] = vi;
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

size_t force_smem(int bpt, int block) { return (size_t)kJSplit * 3 * (block / kJSplit) * bpt * sizeof(float); }

cudaError_t force_prepare(int bpt) {
  static bool done[5] = {};
  if (bpt < 1 || bpt > 4) return cudaErrorInvalidValue;
  if (!done[bpt]) {
    cudaError_t e = cudaFuncSetAttribute(force_fn(bpt), cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    done[bpt] = true;
  }
  return cudaSuccess;
}

cudaError_t launch_nbody_force(const NBodyParams &p, int kick, int bpt, int grid, int block, cudaStream_t s) {
  if (block % (32 * kJSplit) || block > (bpt == 4 ? 512 : 1024)) return cudaErrorInvalidValue;
  cudaError_t e = force_prepare(bpt);
  if (e != cudaSuccess) return e;
  const float hdt = 0.5f * p.dt;
  const size_t sm = force_smem(bpt, block);
  switch (bpt) {
    case 1: force_kernel<1><<<grid, block, sm, s>>>(p.x, p.v, p.a, p.n, p.G, p.eps2, hdt, kick); break;
    case 4: force_kernel<4><<<grid, block, sm, s>>>(p.x, p.v, p.a, p.n, p.G, p.eps2, hdt, kick); break;
    default: force_kernel<2><<<grid, block, sm, s>>>(p.x, p.v, p.a, p.n, p.G, p.eps2, hdt, kick); break;
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
    kp.sharedMemBytes = (unsigned)force_smem(bpt, block);
    kp.kernelParams = args;
    MRW_TRY(force_prepare(bpt));
    MRW_TRY(cudaGraphAddKernelNode(&force_node, body, &drift_node, 1, &kp));
  }
  cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

}  // namespace mrw
