// Fused pointwise chain: a run of consecutive pointwise stages of a Pipeline / Map / MapReduce
// (Section 2.1) evaluated in registers, one HBM read and one HBM write per pixel.
//
// The paper keeps the data a Pipeline's consecutive kernels exchange in device memory, with the
// same partitioning for producer and consumer (Section 3.1, locality-aware domain decomposition).
// On one GPU the partitions are the threads' 16-byte row segments, and consecutive pointwise
// stages share them in registers: no intermediate is materialised.
//
// Thread -> data: a thread owns one 16-byte column segment (16 pixels) of a row and walks down
// the rows with stride `rows_parallel`; grid * block is a multiple of the row's segment count so
// the column stays fixed: the column half of the noise hash is computed once per thread, and only
// the thread owning a row's ragged last segment ever masks bytes. A mirror stage moves no data: it
// flips the column coordinate of the stages after it, and the chain reads its source segment
// reversed (two aligned 16-byte loads and a byte permutation).
//
// Byte arithmetic is SIMD within 32-bit words: solarise flips a byte when its top bit is set; the
// threshold compares bytes without inter-byte borrows; the class counts accumulate in byte lanes
// and are folded into 32-bit counters before a lane can overflow.
//
// MapReduce (Section 2.1; merging function +, Section 3.4) is fused: per-thread counters, warp
// reduction with redux.sync, block reduction in shared memory, and one fire-and-forget 64-bit add
// per block and class into a per-stream set of accumulators; a one-CTA finish kernel, launched
// behind the chain with programmatic dependent launch, sums the sets into the result.
#include "mrw_internal.h"
#include "pixel_ops.cuh"

namespace mrw {
namespace {

__device__ __forceinline__ uint4 ld16(const uint8_t *p) {
  return __ldcs(reinterpret_cast<const uint4 *>(p));
}

// 16 source bytes of output segment [xo, xo+16) for a mirrored chain: output byte k comes from
// source column W-1-xo-k. The source window [s, s+16), s = W-xo-16, starts r = W mod 16 bytes
// past the aligned address a0 = s - r (a0 may be -16 for the row's tail segment, whose first
// aligned vector is then not read). The loads (mirrored_issue) and the byte permutation
// (mirrored_finish) are split so that a row's loads can be in flight while the previous rows are
// computed.
__device__ __forceinline__ void mirrored_issue(const uint8_t *row, int xo, int W, uint4 &lo, uint4 &hi) {
  const int a0 = W - xo - 16 - (W & 15);
  if ((W & 15) == 0) {
    hi = ld16(row + a0);
  } else {
    lo = a0 >= 0 ? ld16(row + a0) : make_uint4(0, 0, 0, 0);
    hi = ld16(row + a0 + 16);
  }
}

__device__ __forceinline__ uint4 mirrored_finish(const uint4 &lo, const uint4 &hi, int W, int q0, uint32_t sel) {
  if ((W & 15) == 0)
    return make_uint4(__byte_perm(hi.w, 0, 0x0123), __byte_perm(hi.z, 0, 0x0123), __byte_perm(hi.y, 0, 0x0123),
                      __byte_perm(hi.x, 0, 0x0123));
  uint32_t w0, w1, w2, w3, w4;
  switch (q0) {
    case 0: w0 = lo.x; w1 = lo.y; w2 = lo.z; w3 = lo.w; w4 = hi.x; break;
    case 1: w0 = lo.y; w1 = lo.z; w2 = lo.w; w3 = hi.x; w4 = hi.y; break;
    case 2: w0 = lo.z; w1 = lo.w; w2 = hi.x; w3 = hi.y; w4 = hi.z; break;
    default: w0 = lo.w; w1 = hi.x; w2 = hi.y; w3 = hi.z; w4 = hi.w; break;
  }
  return make_uint4(__byte_perm(w3, w4, sel), __byte_perm(w2, w3, sel), __byte_perm(w1, w2, sel),
                    __byte_perm(w0, w1, sel));
}

struct Thresh {
  uint32_t t0, t0lo, t1, t1lo;
};

__device__ __forceinline__ Thresh make_thresh(uint32_t t) {
  Thresh h;
  h.t0 = (t & 0xFFu) * 0x01010101u;
  h.t1 = ((t >> 8) & 0xFFu) * 0x01010101u;
  h.t0lo = h.t0 & kLo7;
  h.t1lo = h.t1 & kLo7;
  return h;
}

__device__ __forceinline__ void noise16(uint32_t (&w)[4], const uint32_t (&ch)[16], uint32_t ypre) {
#pragma unroll
  for (int j = 0; j < 4; ++j) w[j] = noise4(w[j], ch[4 * j], ch[4 * j + 1], ch[4 * j + 2], ch[4 * j + 3], ypre);
}

// Applies the chain to U segments: each op is decoded once and applied to all of them, which also
// gives the scheduler U independent dependency chains. Chains with noise stages call it one segment
// at a time (U = 1): their 16 hashes a segment already give the scheduler enough independent work,
// and U segments in flight would exhaust the registers.
template <int NN, int U>
__device__ __forceinline__ void apply_chain(const ChainArgs &a, uint32_t (*w)[4],
                                            const uint32_t (&ch)[NN > 0 ? NN : 1][16], const uint32_t *ypre) {
  // common sequences first: one uniform branch instead of a walk over the op list
  const int pat = a.pattern;
  if (pat == PAT_NONE) return;
  if (pat == PAT_SOLARISE) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < 4; ++j) w[u][j] = solarise4(w[u][j]);
    return;
  }
  if (pat == PAT_THRESH) {
    const Thresh t = make_thresh(a.pattern_t);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < 4; ++j) w[u][j] = (ge4(w[u][j], t.t0, t.t0lo) >> 7) + (ge4(w[u][j], t.t1, t.t1lo) >> 7);
    return;
  }
  if constexpr (NN >= 1) {
    if (pat == PAT_NOISE || pat == PAT_NOISE_SOLARISE) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        noise16(w[u], ch[0], ypre[u]);
        if (pat == PAT_NOISE_SOLARISE)
#pragma unroll
          for (int j = 0; j < 4; ++j) w[u][j] = solarise4(w[u][j]);
      }
      return;
    }
  }
  int kn = 0;
  for (int i = 0; i < a.nops; ++i) {
    const int kind = a.ops[i].kind;
    if (kind == OP_SOLARISE) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j) w[u][j] = solarise4(w[u][j]);
    } else if (kind == OP_THRESH) {
      const Thresh t = make_thresh(a.ops[i].t);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          w[u][j] = (ge4(w[u][j], t.t0, t.t0lo) >> 7) + (ge4(w[u][j], t.t1, t.t1lo) >> 7);
    } else if (kind == OP_NOISE) {
      if constexpr (NN >= 1) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (kn == 0) noise16(w[u], ch[0], ypre[u]);
          if constexpr (NN >= 2) {
            if (kn == 1) noise16(w[u], ch[1], ypre[u]);
          }
        }
      }
      ++kn;
    }
    // OP_MIRROR moves no data: it is folded into the source addressing and the flip flags
  }
}

__device__ __forceinline__ uint32_t byte_sum(uint32_t v) { return __dp4a(v, 0x01010101u, 0u); }

// CTAs per SM the registers of a variant are budgeted for (at most 48 registers for 5, 64 for 4,
// 80 for 3, 128 for 2). Chains with noise keep 16 column hashes per noise op and the next rows'
// loads in registers and are ALU-bound, so their budget follows the unroll depth. Chains without
// noise are HBM-bound: at unroll 4 they fit 48 registers, which lets 5 CTAs of 256 threads (a
// quarter more loads in flight than 4) share an SM; the other depths keep the compiler's choice
// (0: no minimum).
constexpr int chain_min_blocks(int nn, int u) {
  return nn == 0 ? (u == 4 ? 5 : 0) : (nn == 1 ? (u == 1 ? 4 : (u == 2 ? 3 : (u == 4 ? 2 : 1))) : (u <= 2 ? 2 : 1));
}

template <int NN, bool MIR, int U>
__global__ void __launch_bounds__(256, chain_min_blocks(NN, U)) chain_kernel(const __grid_constant__ ChainArgs a) {
  // grid * block <= 2^30 threads (kMaxChainGrid CTAs of at most 256): 32-bit thread indices
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t cv = (uint32_t)a.col_vecs;
  const uint32_t nthreads = (uint32_t)a.rows_parallel * cv;
  // class counts: ge0 = #(label >= 1), ge1 = #(label == 2), n = pixels seen
  uint32_t cnt_ge0 = 0, cnt_ge1 = 0, cnt_n = 0;
  unsigned long long vsum = 0;

  // let the next kernel on the stream be scheduled as soon as SM resources free up
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (gid >= nthreads) asm volatile("griddepcontrol.wait;" ::: "memory");
  if (gid < nthreads) {
    uint32_t col, r0;
    if ((cv & (cv - 1)) == 0) {  // power-of-two segment count (W a multiple of 16 * 2^k)
      col = gid & (cv - 1);
      r0 = gid >> (__ffs(cv) - 1);
    } else {
      r0 = gid / cv;
      col = gid - r0 * cv;
    }
    const int xo = (int)col * 16;
    const int W = a.W;
    const int nv = min(16, W - xo);
    const bool full = nv == 16;
    const int r = W & 15;
    const int q0 = r >> 2, b = r & 3;
    const uint32_t sel = (uint32_t)(b + 3) | ((uint32_t)(b + 2) << 4) | ((uint32_t)(b + 1) << 8) | ((uint32_t)b << 12);

    // Column half of each noise op's hash, c = F(F(seed) ^ x), stored as c ^ (c >> 16): the first
    // xor-shift of F(c ^ y) splits into a column part and a row part.
    uint32_t ch[NN > 0 ? NN : 1][16];
    if constexpr (NN > 0) {
      int kn = 0;
      for (int i = 0; i < a.nops && kn < NN; ++i) {
        if (a.ops[i].kind != OP_NOISE) continue;
        const uint32_t fs = fmix32(a.ops[i].seed);
        const int flip = a.ops[i].flip;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const uint32_t x = flip ? (uint32_t)(W - 1 - xo - k) : (uint32_t)(xo + k);
          const uint32_t c = fmix32(fs ^ x);
          const uint32_t v = c ^ (c >> 16);
          if (kn == 0) ch[0][k] = v;
          if constexpr (NN >= 2) {
            if (kn == 1) ch[1][k] = v;
          }
        }
        ++kn;
      }
    }
    // Programmatic dependent launch: everything above reads only kernel parameters, so it may run
    // while the previous kernel on the stream drains; global memory is touched only after it ends.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // valid-byte masks of this thread's segment (all ones unless it is the row's ragged tail)
    uint32_t vmask[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nb = min(max(nv - 4 * j, 0), 4);
      vmask[j] = nb >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nb)) - 1u);
    }
    // byte-lane counters: lane0 sums the label bytes (n1 + 2 n2), lane1 sums their bit 1 (2 n2);
    // each lane grows by at most 8 a segment
    uint32_t lane0 = 0, lane1 = 0;
    int since_fold = 0;
    // persistent order: rows r0 + (k U + u) step; blocked order: rows (r0 + k step) U + u
    const int64_t step = a.rows_parallel;
    const int64_t ustep = a.blocked ? 1 : step;
    // Chains with noise stages are software-pipelined: the loads of the next U rows are issued
    // before the current U rows are computed, so each warp has a full iteration of hash arithmetic
    // to cover their latency. Chains without noise are HBM-bound and spend their registers on
    // occupancy instead: they load each iteration's rows at its start.
    constexpr bool kAhead = NN > 0;
    uint4 plo[U], phi[U];
    auto issue = [&](int64_t ys) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t y = ys + u * ustep;
        plo[u] = phi[u] = make_uint4(0, 0, 0, 0);
        if (y < a.rows) {
          const uint8_t *row = a.in + y * a.in_pitch;
          if constexpr (MIR) mirrored_issue(row, xo, W, plo[u], phi[u]);
          else phi[u] = ld16(row + xo);
        }
      }
    };
    int64_t y0 = a.blocked ? (int64_t)r0 * U : (int64_t)r0;
    if (kAhead && y0 < a.rows) issue(y0);
    for (; y0 < a.rows; y0 += U * step) {
      uint32_t w[U][4], ypre[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t y = y0 + u * ustep;
        uint4 v = make_uint4(0, 0, 0, 0);
        if constexpr (kAhead) {
          v = MIR ? mirrored_finish(plo[u], phi[u], W, q0, sel) : phi[u];
        } else if (y < a.rows) {
          const uint8_t *row = a.in + y * a.in_pitch;
          if constexpr (MIR) {
            uint4 lo = make_uint4(0, 0, 0, 0), hi;
            mirrored_issue(row, xo, W, lo, hi);
            v = mirrored_finish(lo, hi, W, q0, sel);
          } else {
            v = ld16(row + xo);
          }
        }
        w[u][0] = v.x;
        w[u][1] = v.y;
        w[u][2] = v.z;
        w[u][3] = v.w;
        const uint32_t y32 = (uint32_t)(y + a.row0);
        ypre[u] = y32 ^ (y32 >> 16);
      }
      if (kAhead && y0 + U * step < a.rows) issue(y0 + U * step);
      if constexpr (NN == 0) {
        apply_chain<0, U>(a, w, ch, ypre);
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) apply_chain<NN, 1>(a, &w[u], ch, &ypre[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t y = y0 + u * ustep;
        if (y >= a.rows) break;
        if (a.reduce == RED_COUNT3) {
          // label bytes 0, 1, 2 (a threshold stage's output): with n1, n2 the counts of labels 1
          // and 2, the byte sum is n1 + 2 n2 and the sum of bit 1 is 2 n2
          const uint32_t m0 = w[u][0] & vmask[0], m1 = w[u][1] & vmask[1];
          const uint32_t m2 = w[u][2] & vmask[2], m3 = w[u][3] & vmask[3];
          lane0 += (m0 + m1) + (m2 + m3);
          lane1 += ((m0 & 0x02020202u) + (m1 & 0x02020202u)) + ((m2 & 0x02020202u) + (m3 & 0x02020202u));
          cnt_n += nv;
        } else if (a.reduce == RED_SUM) {
          uint32_t s4 = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) s4 = __dp4a(w[u][j] & vmask[j], 0x01010101u, s4);
          vsum += s4;
        }
        if (a.out) {
          uint8_t *orow = a.out + y * a.out_pitch + xo;
          if (full) {
            __stcs(reinterpret_cast<uint4 *>(orow), make_uint4(w[u][0], w[u][1], w[u][2], w[u][3]));
          } else {
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (k < nv) orow[k] = (uint8_t)(w[u][k >> 2] >> (8 * (k & 3)));
          }
        }
      }
      if (a.reduce == RED_COUNT3 && (since_fold += U) > 31 - U) {  // fold before a lane reaches 256
        cnt_ge0 += byte_sum(lane0);
        cnt_ge1 += byte_sum(lane1);
        lane0 = lane1 = 0;
        since_fold = 0;
      }
    }
    cnt_ge0 += byte_sum(lane0);
    cnt_ge1 += byte_sum(lane1);
    // cnt_ge0 = n1 + 2 n2 and cnt_ge1 = 2 n2 here: make them #(label >= 1) and #(label == 2)
    cnt_ge1 >>= 1;
    cnt_ge0 -= cnt_ge1;
  }

  if (a.reduce == RED_NONE) return;
  __shared__ unsigned long long red_smem[32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long r0v, r1v, r2v;
  if (a.reduce == RED_COUNT3) {
    const uint32_t s0 = __reduce_add_sync(0xFFFFFFFFu, cnt_ge0);
    const uint32_t s1 = __reduce_add_sync(0xFFFFFFFFu, cnt_ge1);
    const uint32_t sn = __reduce_add_sync(0xFFFFFFFFu, cnt_n);
    r0v = (unsigned long long)(sn - s0);  // label 0
    r1v = (unsigned long long)(s0 - s1);  // label 1
    r2v = s1;                             // label 2
  } else {
    unsigned long long s = vsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    r0v = s;
    r1v = r2v = 0;
  }
  if (lane == 0) {
    red_smem[warp][0] = r0v;
    red_smem[warp][1] = r1v;
    red_smem[warp][2] = r2v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int nout = a.reduce == RED_COUNT3 ? 3 : 1;
  unsigned long long t[3] = {0, 0, 0};
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) {
    t[0] += red_smem[i][0];
    t[1] += red_smem[i][1];
    t[2] += red_smem[i][2];
  }
  // with a workspace: add into accumulator set blockIdx % kChainSlots (left at zero by the
  // previous finish), which the finish kernel sums into `red`; without: add into a zeroed `red`.
  // The result of the add is not used, so the CTA does not wait for it.
  unsigned long long *dst = a.partials ? a.partials + 3 * (blockIdx.x % kChainSlots) : a.red;
  for (int k = 0; k < nout; ++k)
    if (t[k]) atomicAdd(dst + k, t[k]);
}

// The MapReduce finish: the kChainSlots accumulator sets of the chain launch before it on the
// stream, summed into `red` and zeroed for the next launch. Launched with programmatic dependent
// launch: griddepcontrol.wait returns once that launch has completed and its adds are visible.
__global__ void __launch_bounds__(kChainSlots) chain_finish_kernel(unsigned long long *partials,
                                                                   unsigned long long *red, int nout) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ unsigned long long s[kChainSlots / 32][3];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  unsigned long long v[3] = {0, 0, 0};
  for (int k = 0; k < nout; ++k) {
    v[k] = __ldcg(partials + 3 * t + k);
    partials[3 * t + k] = 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    for (int k = 0; k < 3; ++k) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], o);
  if (lane == 0)
    for (int k = 0; k < 3; ++k) s[warp][k] = v[k];
  __syncthreads();
  if (t == 0)
    for (int k = 0; k < nout; ++k) {
      unsigned long long tot = 0;
      for (int i = 0; i < kChainSlots / 32; ++i) tot += s[i][k];
      red[k] = tot;
    }
}

template <int NN, bool MIR, int U>
const void *kernel_ptr() {
  return (const void *)chain_kernel<NN, MIR, U>;
}

template <int NN, bool MIR>
const void *pick_u(int unroll) {
  switch (unroll) {
    case 1: return kernel_ptr<NN, MIR, 1>();
    case 2: return kernel_ptr<NN, MIR, 2>();
    case 8: return kernel_ptr<NN, MIR, 8>();
    default: return kernel_ptr<NN, MIR, 4>();
  }
}

const void *pick(int n_noise, bool mir, int unroll) {
  switch (n_noise) {
    case 0: return mir ? pick_u<0, true>(unroll) : pick_u<0, false>(unroll);
    case 1: return mir ? pick_u<1, true>(unroll) : pick_u<1, false>(unroll);
    case 2: return mir ? pick_u<2, true>(unroll) : pick_u<2, false>(unroll);
    default: return nullptr;
  }
}

}  // namespace

int chain_blocks_per_sm(int n_noise, bool mirror, int unroll, int block) {
  static int cache[3][2][4][9] = {};  // [noise][mirror][unroll 1,2,4,8][block / 32, up to 256]
  const int ui = unroll == 1 ? 0 : unroll == 2 ? 1 : unroll == 8 ? 3 : 2;
  const int bi = block / 32;
  if (n_noise < 0 || n_noise > 2 || bi < 1 || bi > 8) return 1;
  int &c = cache[n_noise][mirror ? 1 : 0][ui][bi];
  if (c) return c;
  const void *fn = pick(n_noise, mirror, unroll);
  int nb = 0;
  if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  c = nb > 0 ? nb : 1;
  return c;
}

// Programmatic dependent launch for a launch on `s`, unless `s` is being captured into a graph
// (the graph keeps plain dependencies).
static int pdl_attrs(cudaStream_t s, cudaLaunchAttribute *attr) {
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusNone;
  return cap == cudaStreamCaptureStatusNone ? 1 : 0;
}

cudaError_t launch_chain_finish(unsigned long long *partials, unsigned long long *red, int nout, cudaStream_t s) {
  if (!partials || !red || nout < 1 || nout > 3) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(kChainSlots);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  cfg.attrs = attr;
  cfg.numAttrs = pdl_attrs(s, attr);
  return cudaLaunchKernelEx(&cfg, chain_finish_kernel, partials, red, nout);
}

cudaError_t chain_node(const ChainArgs &ca, int n_noise, int unroll, int grid, int block, NodeChain &nc) {
  if (grid <= 0) return cudaSuccess;
  ChainArgs a = ca;  // copied into the node's parameters by cudaGraphAddKernelNode
  a.pattern = op_pattern(a.ops, a.nops, &a.pattern_t);
  const void *fn = pick(n_noise, a.mirror != 0, unroll);
  if (!fn) return cudaErrorInvalidValue;
  void *args[] = {(void *)&a};
  return nc.kernel(fn, dim3(grid), dim3(block), 0, args);
}

cudaError_t launch_chain(const ChainArgs &ca, int n_noise, int unroll, int grid, int block, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  ChainArgs a = ca;
  a.pattern = op_pattern(a.ops, a.nops, &a.pattern_t);
  const void *fn = pick(n_noise, a.mirror != 0, unroll);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  cfg.attrs = attr;
  cfg.numAttrs = pdl_attrs(s, attr);
  void *args[] = {(void *)&a};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace mrw
