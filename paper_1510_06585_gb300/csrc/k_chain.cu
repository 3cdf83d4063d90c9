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
// the column stays fixed and the column half of the noise hash is computed once per thread.
// A mirror stage moves no data: it flips the column coordinate of the stages after it, and the
// chain reads its source segment reversed (two aligned 16-byte loads and a byte permutation).
//
// MapReduce (Section 2.1; merging function +, Section 3.4) is fused: per-thread counters, warp
// reduction with redux.sync, block reduction in shared memory, one 64-bit atomic per block.
#include "mrw_internal.h"

namespace mrw {
namespace {

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ uint4 ld16(const uint8_t *p) {
  return __ldcs(reinterpret_cast<const uint4 *>(p));
}

// 16 source bytes of output segment [xo, xo+16) for a mirrored chain: output byte k comes from
// source column W-1-xo-k. The source window [s, s+16), s = W-xo-16, starts r = W mod 16 bytes
// past the aligned address a0 = s - r (a0 may be -16 for the row's tail segment, whose first
// aligned vector is then not read).
__device__ __forceinline__ uint4 load_mirrored(const uint8_t *row, int xo, int W, int q0, uint32_t sel) {
  const int s = W - xo - 16;
  const int a0 = s - (W & 15);
  if ((W & 15) == 0) {
    const uint4 v = ld16(row + a0);
    return make_uint4(__byte_perm(v.w, 0, 0x0123), __byte_perm(v.z, 0, 0x0123), __byte_perm(v.y, 0, 0x0123),
                      __byte_perm(v.x, 0, 0x0123));
  }
  const uint4 lo = a0 >= 0 ? ld16(row + a0) : make_uint4(0, 0, 0, 0);
  const uint4 hi = ld16(row + a0 + 16);
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

__device__ __forceinline__ uint32_t solarise4(uint32_t w) {
  // p >= 128 -> 255 - p == p ^ 0xFF; the top bit of each byte selects the flip
  return w ^ (((w >> 7) & 0x01010101u) * 0xFFu);
}

__device__ __forceinline__ uint32_t thresh4(uint32_t w, uint32_t t) {
  const uint32_t t0 = (t & 0xFFu) * 0x01010101u, t1 = ((t >> 8) & 0xFFu) * 0x01010101u;
  return (__vcmpgeu4(w, t0) & 0x01010101u) + (__vcmpgeu4(w, t1) & 0x01010101u);
}

__device__ __forceinline__ uint32_t noise_byte(uint32_t p, uint32_t colhash, uint32_t y) {
  const uint32_t h = fmix32(colhash ^ y);
  const int q = (int)p + (int)(h % 41u) - 20;
  return (uint32_t)min(max(q, 0), 255);
}

__device__ __forceinline__ void noise16(uint32_t (&w)[4], const uint32_t (&ch)[16], uint32_t y) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t b0 = noise_byte(w[j] & 0xFFu, ch[4 * j + 0], y);
    const uint32_t b1 = noise_byte((w[j] >> 8) & 0xFFu, ch[4 * j + 1], y);
    const uint32_t b2 = noise_byte((w[j] >> 16) & 0xFFu, ch[4 * j + 2], y);
    const uint32_t b3 = noise_byte(w[j] >> 24, ch[4 * j + 3], y);
    w[j] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
  }
}

template <int NN>
__device__ __forceinline__ void apply_chain(const ChainArgs &a, uint32_t (&w)[4], const uint32_t (&ch)[NN > 0 ? NN : 1][16],
                                            uint32_t y) {
  int kn = 0;
  for (int i = 0; i < a.nops; ++i) {
    const int kind = a.ops[i].kind;
    if (kind == OP_SOLARISE) {
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = solarise4(w[j]);
    } else if (kind == OP_THRESH) {
      const uint32_t t = a.ops[i].t;
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = thresh4(w[j], t);
    } else if (kind == OP_NOISE) {
      if constexpr (NN >= 1) {
        if (kn == 0) noise16(w, ch[0], y);
        if constexpr (NN >= 2) {
          if (kn == 1) noise16(w, ch[1], y);
        }
      }
      ++kn;
    }
    // OP_MIRROR moves no data: it is folded into the source addressing and the flip flags
  }
}

template <int NN, bool MIR, int U>
__global__ void __launch_bounds__(256) chain_kernel(const __grid_constant__ ChainArgs a) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = a.rows_parallel * a.col_vecs;
  uint32_t c1 = 0, c2 = 0, cn = 0;
  unsigned long long vsum = 0;

  if (gid < nthreads) {
    const int col = (int)(gid % a.col_vecs);
    const int64_t r0 = gid / a.col_vecs;
    const int xo = col * 16;
    const int W = a.W;
    const int nv = min(16, W - xo);
    const int r = W & 15;
    const int q0 = r >> 2, b = r & 3;
    const uint32_t sel = (uint32_t)(b + 3) | ((uint32_t)(b + 2) << 4) | ((uint32_t)(b + 1) << 8) | ((uint32_t)b << 12);

    // Column half of each noise op's hash, F(F(seed) ^ x), for this thread's 16 columns.
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
          const uint32_t v = fmix32(fs ^ x);
          if (kn == 0) ch[0][k] = v;
          if constexpr (NN >= 2) {
            if (kn == 1) ch[1][k] = v;
          }
        }
        ++kn;
      }
    }
    const uint32_t vmask[4] = {nv >= 4 ? 0xFFFFFFFFu : (nv <= 0 ? 0u : (1u << (8 * nv)) - 1u),
                               nv >= 8 ? 0xFFFFFFFFu : (nv <= 4 ? 0u : (1u << (8 * (nv - 4))) - 1u),
                               nv >= 12 ? 0xFFFFFFFFu : (nv <= 8 ? 0u : (1u << (8 * (nv - 8))) - 1u),
                               nv >= 16 ? 0xFFFFFFFFu : (nv <= 12 ? 0u : (1u << (8 * (nv - 12))) - 1u)};
    const int64_t step = a.rows_parallel;
    for (int64_t y0 = r0; y0 < a.rows; y0 += U * step) {
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t y = y0 + u * step;
        if (y < a.rows) {
          const uint8_t *row = a.in + y * a.in_pitch;
          v[u] = MIR ? load_mirrored(row, xo, W, q0, sel) : ld16(row + xo);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t y = y0 + u * step;
        if (y < a.rows) {
          uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
          apply_chain<NN>(a, w, ch, (uint32_t)y);
          if (a.reduce == RED_COUNT3) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              c1 += __popc(w[j] & vmask[j] & 0x01010101u);
              c2 += __popc(w[j] & vmask[j] & 0x02020202u);
            }
            cn += nv;
          } else if (a.reduce == RED_SUM) {
            uint32_t s4 = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) s4 = __dp4a(w[j] & vmask[j], 0x01010101u, s4);
            vsum += s4;
          }
          if (a.out) {
            uint8_t *orow = a.out + y * a.out_pitch + xo;
            if (nv == 16) {
              __stcs(reinterpret_cast<uint4 *>(orow), make_uint4(w[0], w[1], w[2], w[3]));
            } else {
              for (int k = 0; k < nv; ++k) orow[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
            }
          }
        }
      }
    }
  }

  if (a.reduce == RED_NONE) return;
  __shared__ unsigned long long red_smem[32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long r0v, r1v, r2v;
  if (a.reduce == RED_COUNT3) {
    const uint32_t s1 = __reduce_add_sync(0xFFFFFFFFu, c1);
    const uint32_t s2 = __reduce_add_sync(0xFFFFFFFFu, c2);
    const uint32_t sn = __reduce_add_sync(0xFFFFFFFFu, cn);
    r0v = (unsigned long long)(sn - s1 - s2);
    r1v = s1;
    r2v = s2;
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
  if (threadIdx.x == 0) {
    unsigned long long t0 = 0, t1 = 0, t2 = 0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) {
      t0 += red_smem[i][0];
      t1 += red_smem[i][1];
      t2 += red_smem[i][2];
    }
    if (a.reduce == RED_COUNT3) {
      if (t0) atomicAdd(a.red + 0, t0);
      if (t1) atomicAdd(a.red + 1, t1);
      if (t2) atomicAdd(a.red + 2, t2);
    } else if (t0) {
      atomicAdd(a.red, t0);
    }
  }
}

template <int NN, bool MIR>
cudaError_t launch_u(const ChainArgs &a, int unroll, int grid, int block, cudaStream_t s) {
  switch (unroll) {
    case 1: chain_kernel<NN, MIR, 1><<<grid, block, 0, s>>>(a); break;
    case 2: chain_kernel<NN, MIR, 2><<<grid, block, 0, s>>>(a); break;
    case 8: chain_kernel<NN, MIR, 8><<<grid, block, 0, s>>>(a); break;
    default: chain_kernel<NN, MIR, 4><<<grid, block, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_chain(const ChainArgs &a, int n_noise, int unroll, int grid, int block, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  const bool mir = a.mirror != 0;
  switch (n_noise) {
    case 0: return mir ? launch_u<0, true>(a, unroll, grid, block, s) : launch_u<0, false>(a, unroll, grid, block, s);
    case 1: return mir ? launch_u<1, true>(a, unroll, grid, block, s) : launch_u<1, false>(a, unroll, grid, block, s);
    case 2: return mir ? launch_u<2, true>(a, unroll, grid, block, s) : launch_u<2, false>(a, unroll, grid, block, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mrw
