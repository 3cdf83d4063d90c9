// FFT stages (Section 4, FFT pipelined with its inversion): forward and inverse DFTs of N = 65536
// complex float32 values (one 512 KB elementary partitioning unit) per row, several transforms
// fused in one launch with the data kept on chip between them.
//
// Four-step decomposition: the values x[256 a + b] form a 256 x 256 matrix V[a][b] and
//   X[k1 + 256 k2] = sum_b W_256^(b k2) W_N^(b k1) sum_a V[a][b] W_256^(a k1),   W_M = e^(-2 pi i / M)
// that is 256-point transforms down the columns (over a), the twiddle W_N^(b k1), 256-point
// transforms along the rows (over b). Reading the result Y[k1 + 256 k2] as a matrix U[k2][k1]
// gives the same shape again, so transforms chain.
//
// One cluster of C = kFftCluster CTAs per row (8; 4 is also supported): CTA r owns the c = 256 / C
// columns b in [c r, c r + c) of V, and after the row transforms the rows k1 in [c r, c r + c) of
// the result - which are the columns [c r, c r + c) of U. Column transforms are local to a CTA;
// between the two halves of a transform each thread pulls the 32 values its row transforms need
// from the owning CTAs' shared memory (distributed shared memory), between two cluster barriers. A
// following transform starts from shared memory; only the first reads and the last writes HBM.
// With 8 CTAs of 256 threads (64 KB of the row and 32 K registers each) two CTAs share an SM, so
// one cluster's loads, stores and barriers overlap another's arithmetic.
//
// 256-point transforms: half a warp per line, radix 16 x 16. Thread t reads positions t + 16 m,
// does a 16-point DFT (radix 4 x 4 in registers), multiplies by W_256^(t k1), transposes through
// shared memory inside its line, does a second 16-point DFT and writes position t + 16 k2.
//
// Shared-memory layouts (8-byte elements, bank-conflict-free for every access pattern used here):
//   AB (the first transform's input, element (a, j), j = b - c r):
//       a * c + (j ^ ((a ^ (a >> 4)) & 15))
//   BA (everything after the first exchange, element (j, a)):
//       j * 256 + ((a & 0xF0) | ((a ^ (a >> 4) ^ j) & 15))
#include <cooperative_groups.h>

#include <atomic>

#include "fft_ops.cuh"
#include "mrw_internal.h"

namespace cg = cooperative_groups;

namespace mrw {
namespace {

constexpr int kN = kFftN;          // 65536
constexpr int kCols = 256 / kFftCluster;                // columns per CTA (64 or 32)
constexpr int kThreads = kFftCluster == 4 ? 512 : 256;  // half a warp per line, kLines lines at a time
constexpr int kLines = kThreads / 16;                   // lines a CTA transforms at once
constexpr int kUnits = kN / kFftCluster / 2;            // 16-byte units of a CTA's part of a row
constexpr int kMinBlocks = kFftCluster == 4 ? 1 : 2;    // CTAs per SM the registers are budgeted for
static_assert(kFftCluster == 4 || kFftCluster == 8, "clusters of 4 or 8 CTAs");
static_assert(kCols % kLines == 0 && kUnits % kThreads == 0, "whole rounds");

struct FftSmem {
  float2 d[kN / kFftCluster];  // this CTA's part of the row (128 or 64 KB)
  float2 tw[16][16];     // W_256^(t k), stored at [k][t] (forward sign)
  float2 tlo[kCols][16]; // W_N^(b l),      b = kCols r + j, l < 16
  float2 thi[kCols][16]; // W_N^(16 b h),   h < 16
  uint32_t tmem;         // TMEM address of the CTA's 128 columns (the TMEM-stash form)
};

__device__ __forceinline__ int ab(int a, int j) { return a * kCols + (j ^ ((a ^ (a >> 4)) & 15)); }
__device__ __forceinline__ int ba(int j, int a) { return j * 256 + ((a & 0xF0) | ((a ^ (a >> 4) ^ j) & 15)); }

using namespace fftk;  // complex arithmetic and the 16-point DFT

// Shared-memory window address of this CTA's `p` in the CTA of the cluster with rank `rank`, and an
// 8-byte load from such an address (distributed shared memory).
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) from global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

// Tensor memory (TMEM) as a per-thread stash: 32 consecutive 32-bit columns of the thread's lane
// (lane 32 (warp % 4) + laneid, the lanes a warp may reach) hold the 16 complex values of one round.
// tcgen05.st reads its registers when it issues; tcgen05.wait::st / wait::ld wait for the
// thread's own stores / loads to complete.
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float2 (&v)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
               ::"r"(taddr), "r"(__float_as_uint(v[0].x)), "r"(__float_as_uint(v[0].y)), "r"(__float_as_uint(v[1].x)), "r"(__float_as_uint(v[1].y)), "r"(__float_as_uint(v[2].x)), "r"(__float_as_uint(v[2].y)), "r"(__float_as_uint(v[3].x)), "r"(__float_as_uint(v[3].y)), "r"(__float_as_uint(v[4].x)), "r"(__float_as_uint(v[4].y)), "r"(__float_as_uint(v[5].x)), "r"(__float_as_uint(v[5].y)), "r"(__float_as_uint(v[6].x)), "r"(__float_as_uint(v[6].y)), "r"(__float_as_uint(v[7].x)), "r"(__float_as_uint(v[7].y)), "r"(__float_as_uint(v[8].x)), "r"(__float_as_uint(v[8].y)), "r"(__float_as_uint(v[9].x)), "r"(__float_as_uint(v[9].y)), "r"(__float_as_uint(v[10].x)), "r"(__float_as_uint(v[10].y)), "r"(__float_as_uint(v[11].x)), "r"(__float_as_uint(v[11].y)), "r"(__float_as_uint(v[12].x)), "r"(__float_as_uint(v[12].y)), "r"(__float_as_uint(v[13].x)), "r"(__float_as_uint(v[13].y)), "r"(__float_as_uint(v[14].x)), "r"(__float_as_uint(v[14].y)), "r"(__float_as_uint(v[15].x)), "r"(__float_as_uint(v[15].y))
               : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float2 (&v)[16]) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr)
               : "memory");
  // the registers are defined only once the load has completed: every use depends on the wait
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])::"memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}

// Index of line position p in shared memory: a column of the AB layout, or a row of the BA one.
template <bool AB>
__device__ __forceinline__ int line_idx(int line, int p) {
  return AB ? ab(p, line) : ba(line, p);
}

// Pass 1 of a 256-point transform on values already in registers (v[m] = position t + 16 m): the
// 16-point DFT and the W_256^(t k1) twiddle; y[k1] is returned in v[dft16_slot(k1)].
template <int S>
__device__ __forceinline__ void pass1(float2 (&v)[16], int t, const float2 (*tw)[16]) {
  dft16<S>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) {
    const float2 w = conj_if(tw[k1][t], S < 0);
    v[dft16_slot(k1)] = cmul(v[dft16_slot(k1)], w);
  }
}

// Pass 1's output of thread t to positions 16 k1 + t of the line, then pass 2: the 16-point DFTs
// over the rows of the 16 x 16 line matrix. The final value X[t + 16 k2] is multiplied by
// fin(k2) and written to position t + 16 k2.
template <int S, bool AB, class Fin>
__device__ __forceinline__ void pass2(float2 *d, int line, int t, float2 (&v)[16], Fin fin) {
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) d[line_idx<AB>(line, 16 * k1 + t)] = v[dft16_slot(k1)];
  __syncwarp();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) v[n2] = d[line_idx<AB>(line, 16 * t + n2)];
  __syncwarp();
  dft16<S>(v);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) d[line_idx<AB>(line, t + 16 * k2)] = fin(k2, v[dft16_slot(k2)]);
}

// Pass 2 from values already in place: the 16-point DFT over row t of the 16 x 16 line matrix,
// X[t + 16 k2] scaled and written to position t + 16 k2.
template <int S, bool AB>
__device__ __forceinline__ void pass2_in_place(float2 *d, int line, int t, float scale) {
  float2 v[16];
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) v[n2] = d[line_idx<AB>(line, 16 * t + n2)];
  dft16<S>(v);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const float2 x = v[dft16_slot(k2)];
    d[line_idx<AB>(line, t + 16 * k2)] = make_float2(x.x * scale, x.y * scale);
  }
}

// One transform (sign S) of this CTA's part: column transforms (input layout AB or BA), the
// exchange, row transforms into layout BA. Every thread of every CTA of the cluster calls it.
// Between the exchange's pulls and the barrier after them, the pass-1 results wait in registers, or
// with TM in the thread's TMEM columns from `ta` on (32 per round), which frees the registers for a
// third CTA per SM.
template <int S, bool AB, bool TM>
__device__ void transform(FftSmem &sm, cg::cluster_group &cluster, int rank, float scale, uint32_t ta) {
  const int tid = threadIdx.x;
  const int t = tid & 15, g = tid >> 4;  // line group: 32 lines at a time
  float2 *d = sm.d;
  // column transforms over a, with the four-step twiddle W_N^(S b k) folded into the last write
#pragma unroll 1
  for (int line = g; line < kCols; line += kThreads / 16) {
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = d[line_idx<AB>(line, t + 16 * m)];
    pass1<S>(v, t, sm.tw);
    __syncwarp();
    const float2 lo = conj_if(sm.tlo[line][t], S < 0);
    pass2<S, AB>(d, line, t, v, [&](int k2, float2 x) {
      return cmul(x, cmul(lo, conj_if(sm.thi[line][k2], S < 0)));
    });
  }
  cluster.sync();  // every part's column transforms are done
  constexpr int kRounds = kCols / (kThreads / 16);
  // AB: pull the values of this CTA's rows k1 = kCols rank + line for b = t + 16 m from their
  // owners; in layout AB a half warp's 16 values of one line are contiguous in the owner's memory.
  // BA: one value b of 32 consecutive lines is contiguous: a warp pulls for 32 lines at one position
  // tq (one line per lane), so each pull reads whole 32-byte sectors of the owner's memory; the
  // pass-1 results then go to this CTA's rows and pass 2 reads them back with the usual mapping
  // (half a warp per line) after a barrier.
  const int tq = AB ? t : tid / kLines, gq = AB ? g : tid % kLines;
  auto pull = [&](int rd, float2 (&v)[16]) {
    const int k1 = kCols * rank + gq + rd * (AB ? kThreads / 16 : kLines);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int b = tq + 16 * m;  // owned by rank b / kCols = m / (kCols / 16)
      const float2 *src = AB ? d + ab(k1, b & (kCols - 1)) : d + ba(b & (kCols - 1), k1);
      v[m] = ld_cluster(cluster_addr(src, (uint32_t)(m / (kCols / 16))));
    }
    pass1<S>(v, tq, sm.tw);
  };
  auto finish = [&](int rd, float2 (&v)[16]) {
    if constexpr (AB) {
      pass2<S, false>(d, g + rd * (kThreads / 16), t, v, [&](int, float2 x) { return make_float2(x.x * scale, x.y * scale); });
    } else {
      const int line = gq + rd * kLines;
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) d[ba(line, 16 * k1 + tq)] = v[dft16_slot(k1)];
    }
  };
  if constexpr (TM) {
#pragma unroll 1
    for (int rd = 0; rd < kRounds; ++rd) {
      float2 v[16];
      pull(rd, v);
      tm_st16(ta + 32u * (uint32_t)rd, v);
    }
    tm_wait_st();
    cluster.sync();  // every pull is done: the parts may be overwritten
#pragma unroll 1
    for (int rd = 0; rd < kRounds; ++rd) {
      float2 v[16];
      tm_ld16(ta + 32u * (uint32_t)rd, v);
      finish(rd, v);
    }
  } else {
    float2 v[kRounds][16];
#pragma unroll
    for (int rd = 0; rd < kRounds; ++rd) pull(rd, v[rd]);
    cluster.sync();  // every pull is done: the parts may be overwritten
#pragma unroll
    for (int rd = 0; rd < kRounds; ++rd) finish(rd, v[rd]);
  }
  if constexpr (!AB) {
    __syncthreads();
#pragma unroll
    for (int rd = 0; rd < kRounds; ++rd) pass2_in_place<S, false>(d, g + rd * (kThreads / 16), t, scale);
  }
  __syncthreads();
}

// Row r and first column j of the 16-byte unit e (0 .. kUnits - 1) of a CTA's part, for the global
// loads and stores: a warp covers two rows (r even and r + 1) and 32 of their columns (all 32 of
// them in clusters of 8, one half of 64 in clusters of 4), 8 lanes per 128-byte segment; each half
// warp then touches 16 distinct bank pairs in both layouts (the swizzles of rows r and r + 1 differ
// in their lowest bit).
__device__ __forceinline__ void fft_io_slot(int e, int *r, int *j) {
  const int ws = e >> 5, lane = e & 31;
  if constexpr (kCols == 64) {
    *r = 2 * (ws >> 1) + ((lane >> 3) & 1);
    *j = 32 * (ws & 1) + 2 * ((lane & 7) + 8 * (lane >> 4));
  } else {
    *r = 2 * ws + ((lane >> 3) & 1);
    *j = 2 * ((lane & 7) + 8 * (lane >> 4));
  }
}

// TM: the exchange's pass-1 results wait in TMEM (128 columns per CTA, allocated by warp 0 for the
// kernel's lifetime), so a thread needs at most 80 registers and three CTAs share an SM.
template <bool TM>
__global__ void __cluster_dims__(kFftCluster, 1, 1) __launch_bounds__(kThreads, TM ? 3 : kMinBlocks)
    fft_cluster_kernel(const __grid_constant__ FftArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  FftSmem &sm = *reinterpret_cast<FftSmem *>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int64_t cl = blockIdx.x / kFftCluster, ncl = gridDim.x / kFftCluster;
  static_assert(!TM || (kFftCluster == 8 && kThreads == 256), "the TMEM stash is laid out for 8 warps");
  if constexpr (TM) {
    // three CTAs of 128 columns fit the SM's 512 (shared memory and registers admit no fourth), so
    // the allocation never waits
    if (tid < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&sm.tmem)),
                   "r"(128u)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }

  // twiddle tables: W_M^e = (cos(2 pi e / M), -sin(2 pi e / M)), exact integer exponents
  for (int e = tid; e < 256; e += kThreads) {
    const int k = e >> 4, t = e & 15;
    float sn, cs;
    sincospif((float)(t * k) / 128.f, &sn, &cs);
    sm.tw[k][t] = make_float2(cs, -sn);
  }
  for (int i = tid; i < kCols * 16; i += kThreads) {
    const int j = i >> 4, l = i & 15;
    const uint32_t b = (uint32_t)(kCols * rank + j);
    float sn, cs;
    sincospif((float)((b * (uint32_t)l) & (kN - 1)) / (float)(kN / 2), &sn, &cs);
    sm.tlo[j][l] = make_float2(cs, -sn);
    sincospif((float)((b * 16u * (uint32_t)l) & (kN - 1)) / (float)(kN / 2), &sn, &cs);
    sm.thi[j][l] = make_float2(cs, -sn);
  }
  __syncthreads();
  uint32_t ta = 0;  // this thread's TMEM columns: lane 32 (warp % 4) + laneid, 64 columns per warp half
  if constexpr (TM) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int w = tid >> 5;
    ta = sm.tmem + ((uint32_t)(32 * (w & 3)) << 16) + 64u * (uint32_t)(w >> 2);
  }

  for (int64_t f = cl; f < a.nfft; f += ncl) {
    // this CTA's columns of row f: element (a, j) = x[256 a + kCols rank + j], layout AB; two values
    // per 16-byte load
    const float4 *src = reinterpret_cast<const float4 *>(a.in + f * kN + kCols * rank);
    // all of the thread's 16 loads in flight before the first store to shared memory (8 at a time
    // in the 80-register TM form)
    constexpr int kLoads = kUnits / kThreads, kBatch = TM ? 8 : kLoads;
#pragma unroll 1
    for (int i0 = 0; i0 < kLoads; i0 += kBatch) {
      float4 q[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        int r, j;
        fft_io_slot(tid + (i0 + i) * kThreads, &r, &j);
        q[i] = __ldcs(src + 128 * r + (j >> 1));
      }
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        int r, j;
        fft_io_slot(tid + (i0 + i) * kThreads, &r, &j);
        sm.d[ab(r, j)] = make_float2(q[i].x, q[i].y);
        sm.d[ab(r, j + 1)] = make_float2(q[i].z, q[i].w);
      }
    }
    __syncthreads();
    for (int s = 0; s < a.nsteps; ++s) {
      const float scale = a.sign[s] > 0 ? 1.f : 1.f / (float)kN;
      if (s == 0) {
        if (a.sign[0] > 0) transform<1, true, TM>(sm, cluster, rank, scale, ta);
        else transform<-1, true, TM>(sm, cluster, rank, scale, ta);
      } else {
        if (a.sign[s] > 0) transform<1, false, TM>(sm, cluster, rank, scale, ta);
        else transform<-1, false, TM>(sm, cluster, rank, scale, ta);
      }
    }
    // the cluster's next row: its 256 segments of this CTA's kCols columns (8 kCols bytes each) into L2
    // while this row is stored, so that its loads are served from L2
    if (f + ncl < a.nfft)
      for (int r = tid; r < 256; r += kThreads)
        prefetch_l2(a.in + (f + ncl) * kN + 256 * r + kCols * rank, (uint32_t)(8 * kCols));
    // element (j, a) of layout BA is y[256 a + kCols rank + j]; two values per 16-byte store
    float4 *dst = reinterpret_cast<float4 *>(a.out + f * kN + kCols * rank);
#pragma unroll 4
    for (int e = tid; e < kUnits; e += kThreads) {
      int r, j;
      fft_io_slot(e, &r, &j);
      const float2 lo = sm.d[ba(j, r)], hi = sm.d[ba(j + 1, r)];
      __stcs(dst + 128 * r + (j >> 1), make_float4(lo.x, lo.y, hi.x, hi.y));
    }
    __syncthreads();
  }
  if constexpr (TM) {
    // every thread's TMEM loads completed (tcgen05.wait::ld in tm_ld16) before the columns go back
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem), "r"(128u) : "memory");
  }
}

// Residency of the TM form: an empty kernel of the same cluster shape, block size, register budget
// (three CTAs per SM) and shared memory. The occupancy calculator counts a kernel that uses tcgen05
// instructions as one CTA per SM, but the hardware places three of these per SM (measured: 51
// clusters resident at once, the figure below, and a 52nd queues); what limits them is shared
// memory and registers, and their 3 x 128 TMEM columns fit the SM's 512.
__global__ void __cluster_dims__(kFftCluster, 1, 1) __launch_bounds__(kThreads, 3) fft_tm_residency_probe() {}

// ---- Clusters of 16 CTAs; the transposes are bulk copies between the CTAs' shared memory ----
//
// CTA r of a row's cluster owns the 16 columns b in [16 r, 16 r + 16) of V for the column
// transforms and the 16 rows k1 in [16 r, 16 r + 16) of the result for the row transforms. Its two
// 32 KB buffers hold 16 lines of 256 values in the line layout li(l, p); after a column phase the
// CTA rewrites its values in the send layout, where the 2 KB block d holds what CTA d's row phase
// needs from it, and 16 bulk copies (cp.async.bulk shared::cluster, completing on the receiver's
// mbarrier) deliver block d into CTA d's other buffer, at the sender's slot: exactly the line
// layout of the receiver's 16 rows. No thread waits on a remote load; one cluster barrier per
// transform makes sure every receive buffer is free before the copies start. With 70 KB of shared
// memory and 256 threads a CTA, three CTAs share an SM.
namespace c16 {
constexpr int kC = 256 / kFft16Cluster;      // 16 lines per CTA
constexpr int kT = 256;                      // 16 threads per line, all lines at once
constexpr int kE = kN / kFft16Cluster;       // 4096 values per CTA
constexpr uint32_t kBlock = kE / kFft16Cluster * 8;  // 2 KB per destination
constexpr uint32_t kPolls = 1u << 22;
static_assert(kC == 16 && kT == 16 * kC, "one round of 16 lines");

struct Smem {
  float2 buf[2][kE];
  float2 tw[16][16];   // W_256^(t k), stored at [k][t] (forward sign)
  float2 tlo[kC][16];  // W_N^(b l),    b = 16 r + j
  float2 thi[kC][16];  // W_N^(16 b h)
  uint64_t bar[2];     // receive barrier of each buffer
};

// Line layout: position p of line l is in 16-value block p >> 4 (the sending CTA's rank, for
// received values), row l of it, column (p ^ l ^ (p >> 4)) & 15: every access pattern below
// touches 16 distinct bank pairs per half warp.
__device__ __forceinline__ int li(int l, int p) { return ((p >> 4) << 8) | (l << 4) | ((p ^ l ^ (p >> 4)) & 15); }
// Send layout of CTA `rank`: the value for destination d, row k of d's lines, from this CTA's line j.
__device__ __forceinline__ int si(int d, int k, int j, int rank) { return (d << 8) | (k << 4) | ((j ^ k ^ rank) & 15); }

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t remote(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, uint32_t polls) {
  for (uint32_t i = 0; i < polls; ++i)
    if (try_wait(bar, parity)) return true;
  return false;
}

// Pass 2 inside line l of buffer d: the pass-1 results v (y[k1] in v[dft16_slot(k1)]) to positions
// 16 k1 + t, then the 16-point DFT of positions 16 t .. 16 t + 15 left in v.
template <int S>
__device__ __forceinline__ void pass2_line(float2 *d, int l, int t, float2 (&v)[16]) {
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) d[li(l, 16 * k1 + t)] = v[dft16_slot(k1)];
  __syncwarp();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) v[n2] = d[li(l, 16 * t + n2)];
  __syncwarp();
  dft16<S>(v);
}

// One transform of the row: column phase on buffer w, exchange into buffer 1 - w of every CTA of
// the cluster, row phase there. Every thread of every CTA calls it. `parity` holds the next
// completion parity of each receive barrier; `failed` records a wait that gave up.
template <int S>
__device__ void transform16(Smem &sm, int w, int rank, float scale, uint32_t &parity, uint32_t polls, bool &failed) {
  const int tid = threadIdx.x, t = tid & 15, l = tid >> 4;
  float2 *d = sm.buf[w];
  float2 *e = sm.buf[1 - w];
  float2 v[16];
  // column transform of line l (column b = 16 rank + l of V) over its 256 positions a
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = d[li(l, t + 16 * m)];
  pass1<S>(v, t, sm.tw);
  __syncwarp();
  pass2_line<S>(d, l, t, v);
  __syncthreads();  // every line has read its values: the buffer takes the send layout
  {
    const float2 lo = conj_if(sm.tlo[l][t], S < 0);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2)  // result k1 = t + 16 k2 goes to CTA k2, row t there
      d[si(k2, t, l, rank)] = cmul(v[dft16_slot(k2)], cmul(lo, conj_if(sm.thi[l][k2], S < 0)));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the copies read these values
  __syncthreads();
  if (tid == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&sm.bar[1 - w])),
                 "r"((uint32_t)kE * 8u)
                 : "memory");
  // every CTA's receive buffer is free (its previous contents were read or stored) and armed
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  if (tid < kFft16Cluster) {  // thread k sends block k to CTA k, into the slot of this CTA
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        "cp.async.bulk.commit_group;" ::"r"(remote(e + (rank << 8), (uint32_t)tid)),
        "r"(saddr(d + (tid << 8))), "r"(kBlock), "r"(remote(&sm.bar[1 - w], (uint32_t)tid))
        : "memory");
  }
  const uint32_t par = (parity >> (1 - w)) & 1u;
  if (!wait_bounded(&sm.bar[1 - w], par, polls)) failed = true;
  parity ^= 1u << (1 - w);
  if (tid < kFft16Cluster) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  __syncthreads();  // the sends have been read: buffer w may be refilled
  // row transform of line l (row k1 = 16 rank + l) over its 256 positions b
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = e[li(l, t + 16 * m)];
  pass1<S>(v, t, sm.tw);
  __syncwarp();
  pass2_line<S>(e, l, t, v);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const float2 x = v[dft16_slot(k2)];
    e[li(l, t + 16 * k2)] = make_float2(x.x * scale, x.y * scale);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kT, 3) fft16_kernel(const __grid_constant__ FftArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int64_t cl = blockIdx.x / kFft16Cluster, ncl = gridDim.x / kFft16Cluster;
  const uint32_t polls = a.wait_polls ? a.wait_polls - 1 : kPolls;

  for (int i = tid; i < 256; i += kT) {
    const int k = i >> 4, t = i & 15;
    float sn, cs;
    sincospif((float)(t * k) / 128.f, &sn, &cs);
    sm.tw[k][t] = make_float2(cs, -sn);
    const uint32_t b = (uint32_t)(kC * rank + k);  // line k, index t
    sincospif((float)((b * (uint32_t)t) & (kN - 1)) / (float)(kN / 2), &sn, &cs);
    sm.tlo[k][t] = make_float2(cs, -sn);
    sincospif((float)((b * 16u * (uint32_t)t) & (kN - 1)) / (float)(kN / 2), &sn, &cs);
    sm.thi[k][t] = make_float2(cs, -sn);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&sm.bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&sm.bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster.sync();  // the barriers exist before any CTA sends

  uint32_t parity = 0;
  bool failed = false;
  for (int64_t f = cl; f < a.nfft; f += ncl) {
    // columns [16 rank, 16 rank + 16) of row f: value (a, j) = x[256 a + 16 rank + j] to line j,
    // position a; two values per 16-byte load, all of a thread's loads in flight first
    {
      const float4 *src = reinterpret_cast<const float4 *>(a.in + f * kN + kC * rank);
      constexpr int kLoads = kE / 2 / kT;
      float4 q[kLoads];
#pragma unroll
      for (int i = 0; i < kLoads; ++i) {
        const int u = tid + i * kT;
        q[i] = __ldcs(src + 128 * (u >> 3) + (u & 7));
      }
#pragma unroll
      for (int i = 0; i < kLoads; ++i) {
        const int u = tid + i * kT, ar = u >> 3, j = 2 * (u & 7);
        sm.buf[0][li(j, ar)] = make_float2(q[i].x, q[i].y);
        sm.buf[0][li(j + 1, ar)] = make_float2(q[i].z, q[i].w);
      }
    }
    __syncthreads();
    int w = 0;
    for (int s = 0; s < a.nsteps; ++s) {
      const float scale = a.sign[s] > 0 ? 1.f : 1.f / (float)kN;
      if (a.sign[s] > 0) transform16<1>(sm, w, rank, scale, parity, polls, failed);
      else transform16<-1>(sm, w, rank, scale, parity, polls, failed);
      w = 1 - w;
    }
    // line l of buffer w is row k1 = 16 rank + l of the result: y[k1 + 256 p] for positions p,
    // the 16 lines of one position being 128 contiguous bytes; two values per 16-byte store
    {
      float4 *dst = reinterpret_cast<float4 *>(a.out + f * kN + kC * rank);
      const float2 *b = sm.buf[w];
#pragma unroll 4
      for (int u = tid; u < kE / 2; u += kT) {
        const int p = u >> 3, l = 2 * (u & 7);
        const float2 lo = b[li(l, p)], hi = b[li(l + 1, p)];
        __stcs(dst + 128 * p + (u & 7), make_float4(lo.x, lo.y, hi.x, hi.y));
      }
    }
    __syncthreads();
  }
  if (tid < kFft16Cluster) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (failed && a.status) *(volatile unsigned int *)a.status = 1u;
  cluster.sync();  // no CTA leaves while a copy into it could still be under way
}
}  // namespace c16

}  // namespace

size_t fft16_smem_bytes() { return sizeof(c16::Smem); }

int fft16_max_clusters() {
  static int cached = -1;
  if (cached >= 0) return cached;
  int n = 0;
  if (cudaFuncSetAttribute(c16::fft16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(c16::Smem)) == cudaSuccess &&
      cudaFuncSetAttribute(c16::fft16_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(c16::kT);
    cfg.gridDim = dim3(kFft16Cluster);
    cfg.dynamicSmemBytes = sizeof(c16::Smem);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kFft16Cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)c16::fft16_kernel, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  cached = n;
  return n;
}

cudaError_t launch_fft16(const FftArgs &a, int clusters, cudaStream_t s) {
  if (a.nsteps < 1 || a.nsteps > kFftMaxSteps || a.nfft < 1 || clusters < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(c16::fft16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(c16::Smem));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(c16::fft16_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(c16::kT);
  cfg.gridDim = dim3(kFft16Cluster * clusters);
  cfg.dynamicSmemBytes = sizeof(c16::Smem);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kFft16Cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, c16::fft16_kernel, a);
}

size_t fft_smem_bytes() { return sizeof(FftSmem); }

int fft_max_clusters(bool tm) {
  static std::atomic<int> cached[2] = {-1, -1};
  std::atomic<int> &c = cached[tm ? 1 : 0];
  if (c.load() >= 0) return c.load();
  const void *fn = tm ? (const void *)fft_cluster_kernel<true> : (const void *)fft_cluster_kernel<false>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FftSmem)) != cudaSuccess ||
      (tm && cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.gridDim = dim3(kFftCluster);
  cfg.dynamicSmemBytes = sizeof(FftSmem);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) n = 0;
  if (tm && n > 0) {
    // the probe's residency, provided the kernel's own registers admit three CTAs per SM
    cudaFuncAttributes fa{};
    int np = 0;
    const void *probe = (const void *)fft_tm_residency_probe;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.numRegs * kThreads * 3 <= 65536 &&
        cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FftSmem)) == cudaSuccess &&
        cudaFuncSetAttribute(probe, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&np, probe, &cfg) == cudaSuccess && np > n)
      n = np;
  }
  cudaGetLastError();
  c.store(n);
  return n;
}

cudaError_t launch_fft(const FftArgs &a, int clusters, bool tm, cudaStream_t s) {
  if (a.nsteps < 1 || a.nsteps > kFftMaxSteps || a.nfft < 1 || clusters < 1) return cudaErrorInvalidValue;
  const void *fn = tm ? (const void *)fft_cluster_kernel<true> : (const void *)fft_cluster_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FftSmem));
  if (e == cudaSuccess && tm)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (tm) fft_cluster_kernel<true><<<dim3(kFftCluster * clusters), dim3(kThreads), sizeof(FftSmem), s>>>(a);
  else fft_cluster_kernel<false><<<dim3(kFftCluster * clusters), dim3(kThreads), sizeof(FftSmem), s>>>(a);
  return cudaGetLastError();
}

}  // namespace mrw
