// FFT stages (Section 4, FFT pipelined with its inversion) with the four-step transposes exchanged
// through a ring of rows in global memory that stays in the 129 MB L2, instead of through the
// distributed shared memory of a cluster.
//
// Four-step decomposition of one row of N = 65536 values, read as the 256 x 256 matrix
// M[a][b] = x[256 a + b]:
//   forward from natural order (decimation in time):
//     Y[k1][b] = W_N^(S b k1) sum_a M[a][b] W_256^(S a k1)          (down the columns, then twiddle)
//     T[k1][k2] = sum_b Y[k1][b] W_256^(S b k2) = X[k1 + 256 k2]     (along the lines)
//   from that transposed order back to natural order (decimation in frequency):
//     U[k1][n2] = W_N^(S n2 k1) sum_k2 T[k1][k2] W_256^(S n2 k2)     (along the lines, then twiddle)
//     x[256 n1 + n2] = sum_k1 U[k1][n2] W_256^(S n1 k1)              (down the columns)
// with W_M = e^(-2 pi i / M), S = +1 forward and -1 inverse (the inverse also divides by N). The
// transforms of a chain alternate between the two forms, so the line half of transform q and the
// line half of transform q + 1 act on the same lines, and so do their column halves: a chain of
// n transforms is n + 1 phases, column phases and line phases in turn. Phase p holds the second
// half of transform p and the first half of transform p + 1; the first phase reads the input rows,
// the last writes the output rows (a chain of odd length ends on lines, and its last phase writes
// the transposed result back in natural order through shared memory).
//
// Work items: phase p of row f is 16 items of 16 columns (column phases) or 16 lines (line phases),
// 4096 values each, one CTA of 256 threads per item (four CTAs per SM). Between phases a row's
// values wait in its slot of the ring; an item's 32 KB is read and written in 128-byte pieces per
// half warp. Each CTA of a persistent grid claims tickets from a global counter; the ticket order
// puts phase p of a slice of rows L steps after phase p - 1, so an item's inputs are usually
// complete when it is claimed, and a per-row, per-phase completion counter (acquire / release, a
// bounded wait) guards the rest. Every dependency of a ticket lies on a smaller ticket, claimed by
// a running CTA, so the grid always progresses. The last phase of a row discards its ring lines
// from L2 after reading them, so dead values are never written back to HBM. HBM traffic is the
// input read once and the output written once; the four-step twiddles come from a per-device
// 256 x 256 table that stays in L2.
//
// A 256-point DFT is two 16-point DFTs in registers (radix 4 x 4, the 4-point butterflies in paired
// f32x2 instructions) with one transpose through shared memory: in column items across the CTA's
// 8 warps, in line items inside a half warp's line.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "fft_ops.cuh"
#include "mrw_internal.h"

namespace mrw {

// ---- ticket schedule (host and device) ---------------------------------------------------------
// Rows are taken in slices of G. Step s holds phase p of slice s - p L for every p with
// 0 <= s - p L < nslices, in ascending p; a (phase, slice) pair is kFftL2Items G tickets (row-major, then the
// kFftL2Items items of the row). L <= nslices, so every step holds at least one pair.
__host__ __device__ inline int64_t fsch_tri(int64_t v, int64_t L) {  // sum_{u < v} (floor(u / L) + 1)
  if (v <= 0) return 0;
  const int64_t q = v / L, r = v % L;
  return L * q * (q + 1) / 2 + r * (q + 1);
}
__host__ __device__ inline int64_t fsch_steps(const FftSched &c) { return c.nslices + (int64_t)(c.P - 1) * c.L; }
// first phase present in step s
__host__ __device__ inline int64_t fsch_plo(const FftSched &c, int64_t s) {
  return s < c.nslices ? 0 : (s - c.nslices) / c.L + 1;
}
// (phase, slice) pairs in the steps before s
__host__ __device__ inline int64_t fsch_pairs_before(const FftSched &c, int64_t s) {
  const int64_t cap = (int64_t)(c.P - 1) * c.L;
  const int64_t hi = s <= cap ? fsch_tri(s, c.L) : fsch_tri(cap, c.L) + (s - cap) * c.P;
  return hi - fsch_tri(s - c.nslices, c.L);
}
__host__ __device__ inline int64_t fsch_total(const FftSched &c) { return c.nslices * c.G * kFftL2Items * c.P; }
__host__ __device__ inline void fsch_decode(const FftSched &c, int64_t T, int *p, int64_t *f, int *j) {
  const int64_t per = (int64_t)kFftL2Items * c.G, k = T / per, rem = T % per;
  int64_t lo = 0, hi = fsch_steps(c) - 1;  // the last step with pairs_before(s) <= k
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (fsch_pairs_before(c, mid) <= k) lo = mid;
    else hi = mid - 1;
  }
  const int pp = (int)(fsch_plo(c, lo) + (k - fsch_pairs_before(c, lo)));
  *p = pp;
  *f = (lo - (int64_t)pp * c.L) * c.G + rem / kFftL2Items;
  *j = (int)(rem % kFftL2Items);
}
// The same mapping in 32-bit arithmetic without a search in the steady state (every phase present):
// there pairs_before(s) = tri(cap) + (s - cap) P, so the step follows from one division; in the first
// and last (P - 1) L steps a scan of at most (P - 1) L steps finds it. L is 1 or 2, T < 2^31.
__host__ __device__ inline uint32_t fsch_tri32(uint32_t v, uint32_t L) {
  const uint32_t q = v >> (L - 1), r = v & (L - 1);
  return L * q * (q + 1) / 2 + r * (q + 1);
}
__host__ __device__ inline uint32_t fsch_pairs32(const FftSched &c, uint32_t s) {
  const uint32_t L = (uint32_t)c.L, cap = (uint32_t)(c.P - 1) * L, ns = (uint32_t)c.nslices;
  const uint32_t hi = s <= cap ? fsch_tri32(s, L) : fsch_tri32(cap, L) + (s - cap) * (uint32_t)c.P;
  return hi - (s > ns ? fsch_tri32(s - ns, L) : 0u);
}
__host__ __device__ inline void fsch_decode32(const FftSched &c, uint32_t T, int *p, int64_t *f, int *j) {
  const uint32_t per = (uint32_t)kFftL2Items * (uint32_t)c.G, k = T / per, rem = T - k * per;
  const uint32_t L = (uint32_t)c.L, P = (uint32_t)c.P, cap = (P - 1) * L, ns = (uint32_t)c.nslices;
  const uint32_t tcap = fsch_tri32(cap, L);
  uint32_t s = 0;
  if (cap <= ns && k >= tcap) {
    s = cap + (k - tcap) / P;
    if (s > ns) s = ns;
  }
  while (fsch_pairs32(c, s + 1) <= k) ++s;
  const uint32_t plo = s < ns ? 0u : (s - ns) / L + 1;
  const uint32_t pp = plo + (k - fsch_pairs32(c, s));
  *p = (int)pp;
  *f = (int64_t)(s - pp * L) * c.G + rem / kFftL2Items;
  *j = (int)(rem % kFftL2Items);
}
__host__ __device__ inline int64_t fsch_ticket(const FftSched &c, int p, int64_t f, int j) {
  const int64_t sl = f / c.G, s = sl + (int64_t)p * c.L;
  return (fsch_pairs_before(c, s) + (p - fsch_plo(c, s))) * kFftL2Items * c.G + (f - sl * c.G) * kFftL2Items + j;
}

namespace {
using namespace fftk;

constexpr int kN = kFftN;
constexpr int kB = kFftL2Block;  // columns of a column item, lines of a line item
constexpr int kT = 16 * kB;       // threads per CTA: 16 per column or line
constexpr int kJ = kFftL2Items;   // items per row and phase
constexpr uint32_t kPolls = 1u << 21;

constexpr int kLine = 16 * 17;  // a line's 256 values between its two 16-point DFTs, rows padded to 17

struct Smem {
  float2 d[kB * kLine];  // the item's values between the two 16-point DFTs (34 KB)
  float2 tw[16][16];     // W_256^(t k) at [k][t], forward sign
};

__device__ __forceinline__ void reorder(float2 (&v)[16]) {
  float2 t[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = v[dft16_slot(k)];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = t[k];
}

// The output of a 256-point DFT times the four-step twiddles post[k * stride] (TW), whose loads are
// issued once the first 16-point DFT's values have gone to shared memory, so that they travel
// while the second one runs.
template <bool TW>
struct Post {
  const float2 *p;
  int stride;
  float2 v[TW ? 16 : 1];
  __device__ __forceinline__ void load() {
    if constexpr (TW) {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = __ldg(p + k * stride);
    }
  }
  __device__ __forceinline__ void apply(float2 (&x)[16]) const {
    if constexpr (TW) {
#pragma unroll
      for (int k = 0; k < 16; ++k) x[k] = cmul(x[k], v[k]);
    }
  }
};

// 256-point DFT (sign S) down the item's kB columns. Thread (w, lane) holds in v[m] row w + 16 m of
// column lane; on return v[k] holds output row w + 16 k. Layout of d between the two 16-point
// DFTs: [o_lo][w][lane], a half warp's 16 values contiguous in every access.
// Fresh: the item's first transform (the barriers between items already order the buffer's
// previous contents before it).
template <int S, bool TW, bool Fresh>
__device__ __forceinline__ void col_dft(float2 (&v)[16], const Smem &sm, float2 *d, int w, int lane, Post<TW> post) {
  dft16<S>(v);  // over m: output o_lo in v[dft16_slot(o_lo)]
  if constexpr (!Fresh) __syncthreads();  // the buffer's previous contents have been read
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    float2 z = v[dft16_slot(k)];
    if (k) z = cmul(z, conj_if(sm.tw[k][w], S < 0));
    d[(k * 16 + w) * kB + lane] = z;
  }
  post.load();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = d[(w * 16 + i) * kB + lane];
  dft16<S>(v);  // over the first index: output o_hi
  reorder(v);
  post.apply(v);
}

// 256-point DFT (sign S) along one line per half warp. Thread t holds in v[m] position t + 16 m; on
// return v[k] holds output position t + 16 k. The line's 256 values in dl: [o_lo][i], rows of 17
// (the padding keeps both the row writes and the column reads free of bank conflicts, with the
// offsets immediate).
template <int S, bool TW>
__device__ __forceinline__ void row_dft(float2 (&v)[16], const Smem &sm, float2 *dl, int t, Post<TW> post) {
  dft16<S>(v);
  __syncwarp();  // the line's previous contents have been read
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    float2 z = v[dft16_slot(k)];
    if (k) z = cmul(z, conj_if(sm.tw[k][t], S < 0));
    dl[k * 17 + t] = z;
  }
  post.load();
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = dl[t * 17 + i];
  dft16<S>(v);
  reorder(v);
  post.apply(v);
}

__device__ __forceinline__ bool wait_count(const unsigned int *c, unsigned int want, uint32_t polls) {
  for (uint32_t i = 0;; ++i) {
    unsigned int x;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(x) : "l"(c) : "memory");
    if (x >= want) return true;
    if (i >= polls) return false;
    __nanosleep(128);
  }
}
__device__ __forceinline__ void discard_l2(const void *p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
struct Work {
  int64_t f;
  int p, j;
};

// The row of a work item that its copies read: the input row for phase 0, else the row's ring slot.
__device__ __forceinline__ const float2 *item_src(const FftL2Args &a, const Work &wk) {
  return wk.p == 0 ? a.in + wk.f * kN : a.ring + (wk.f % a.ring_rows) * kN;
}

// One column item: columns [kB j, kB j + kB) of row f in phase p (p even). The phase holds the
// column half of transform p (decimation in frequency, sign index p - 1) and the column half of
// transform p + 1 (decimation in time, sign index p) with its twiddle W_N^(S b k1).
__device__ __forceinline__ void col_item(const FftL2Args &a, Smem &sm, const Work &wk, float2 *d) {
  const int tid = threadIdx.x, w = tid / kB, lane = tid % kB;
  const int p = wk.p, j = wk.j;
  const int b = kB * j + lane;
  const bool last = p == a.nsteps, has2 = p >= 1, has1 = p < a.nsteps;
  const int s2 = has2 ? a.sign[p - 1] : 1, s1 = has1 ? a.sign[p] : 1;
  const float2 *src = item_src(a, wk) + b;
  float2 v[16];
  if (p == 0) {
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = __ldcs(src + (w + 16 * m) * 256);
  } else {
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = __ldcg(src + (w + 16 * m) * 256);
  }
  if (has2) {
    if (s2 > 0) col_dft<1, false, true>(v, sm, d, w, lane, Post<false>{});
    else col_dft<-1, false, true>(v, sm, d, w, lane, Post<false>{});
  }
  if (last)  // every thread's loads were consumed before the barriers above: drop the ring lines
    for (int r = tid; r < 256; r += kT) discard_l2(item_src(a, wk) + r * 256 + kB * j);  // from L2 unwritten
  if (has1) {
    // W_N^(S k1 b) at [k1][b], k1 = w + 16 k
    const Post<true> tw{(s1 > 0 ? a.twiddle : a.twiddle + kN) + w * 256 + b, 16 * 256, {}};
    if (has2) {
      if (s1 > 0) col_dft<1, true, false>(v, sm, d, w, lane, tw);
      else col_dft<-1, true, false>(v, sm, d, w, lane, tw);
    } else {
      if (s1 > 0) col_dft<1, true, true>(v, sm, d, w, lane, tw);
      else col_dft<-1, true, true>(v, sm, d, w, lane, tw);
    }
  }
  if (last) {
    float2 *dst = a.out + wk.f * kN + b;
#pragma unroll
    for (int k = 0; k < 16; ++k) __stcs(dst + (w + 16 * k) * 256, v[k]);
  } else {
    float2 *dst = a.ring + (wk.f % a.ring_rows) * kN + b;
#pragma unroll
    for (int k = 0; k < 16; ++k) __stcg(dst + (w + 16 * k) * 256, v[k]);
  }
}

// The last phase of an odd chain: line l = kB j + h holds X[l + 256 k2] at k2 = t + 16 k; transposed
// through shared memory so that a half warp stores 16 consecutive values.
__device__ __forceinline__ void row_last_store(const FftL2Args &a, const Work &wk, float2 *d, const float2 (&v)[16]) {
  const int tid = threadIdx.x, h = tid >> 4, t = tid & 15;
  __syncthreads();  // every line is done with the buffer, and every load has been consumed
  for (int i = tid; i < kB * 16; i += kT)  // drop the item's ring lines from L2 unwritten
    discard_l2(item_src(a, wk) + (int64_t)kB * wk.j * 256 + i * 16);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int k2 = t + 16 * k;
    d[k2 * kB + (h ^ (k2 & (kB - 1)))] = v[k];
  }
  __syncthreads();
  const int w = tid / kB, lane = tid % kB;
  float2 *dst = a.out + wk.f * kN + kB * wk.j + lane;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int k2 = w + 16 * m;
    __stcs(dst + 256 * k2, d[k2 * kB + (lane ^ (k2 & (kB - 1)))]);
  }
}

// One line item: lines [kB j, kB j + kB) of row f's ring slot in phase p (p odd), a half warp per
// line, its values in d as [line][position]. The phase holds the line half of transform p
// (decimation in time, sign index p - 1) and the line half of transform p + 1 (decimation in
// frequency, sign index p) with its twiddle W_N^(S n2 k1). A last phase writes X[l + 256 k2] in
// natural order through shared memory.
template <bool Odd>
__device__ __forceinline__ void row_item(const FftL2Args &a, Smem &sm, const Work &wk, float2 *d) {
  const int tid = threadIdx.x, h = tid >> 4, t = tid & 15;
  const int p = wk.p, j = wk.j;
  const int l = kB * j + h;
  const bool last = p == a.nsteps, has1 = p < a.nsteps;
  const int s2 = a.sign[p - 1], s1 = has1 ? a.sign[p] : 1;
  float2 *dl = d + h * kLine;
  const float2 *src = item_src(a, wk) + (int64_t)l * 256 + t;
  float2 v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = __ldcg(src + 16 * m);
  if (s2 > 0) row_dft<1>(v, sm, dl, t, Post<false>{});
  else row_dft<-1>(v, sm, dl, t, Post<false>{});
  if (has1) {
    // W_N^(S l n2) at [l][n2], n2 = t + 16 k
    const Post<true> tw{(s1 > 0 ? a.twiddle : a.twiddle + kN) + (int64_t)l * 256 + t, 16, {}};
    if (s1 > 0) row_dft<1>(v, sm, dl, t, tw);
    else row_dft<-1>(v, sm, dl, t, tw);
  }
  if (!last) {
    float2 *dst = a.ring + (wk.f % a.ring_rows) * kN + (int64_t)l * 256 + t;
#pragma unroll
    for (int k = 0; k < 16; ++k) __stcg(dst + 16 * k, v[k]);
    return;
  }
  if constexpr (Odd) row_last_store(a, wk, d, v);  // only an odd chain ends on lines
}

// Thread 0: the work item of ticket `t`, claiming further tickets past those that name no row
// (the last slice's missing rows); p = -1 once the tickets are used up.
__device__ Work take(const FftL2Args &a, uint32_t t, uint32_t total) {
  Work wk{0, -1, 0};
  for (;;) {
    if (t >= total) return Work{0, -1, 0};
    fsch_decode32(a.sc, t, &wk.p, &wk.f, &wk.j);
    if (wk.f < a.sc.nfft) return wk;
    t = atomicAdd(a.ticket, 1u);
  }
}
// The completion count that a work item waits for: the row's previous phase, or for phase 0 the
// last phase of the row that held the same ring slot before. Null if there is none.
__device__ __forceinline__ const unsigned int *dep_of(const FftL2Args &a, const Work &wk) {
  const int P = a.sc.P;
  if (wk.p > 0) return a.done + wk.f * P + (wk.p - 1);
  if (wk.f >= a.ring_rows) return a.done + (wk.f - a.ring_rows) * P + (P - 1);
  return nullptr;
}
// Odd: the chain has an odd number of transforms, so its last phase is a line phase (the even
// chains' kernel leaves that path out, which relieves its registers).
template <bool Odd>
__global__ void __launch_bounds__(kT, 4) fft_l2_kernel(const __grid_constant__ FftL2Args a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  __shared__ Work work[2];
  const int tid = threadIdx.x;
  // W_256^(t k) = (cos(2 pi t k / 256), -sin(2 pi t k / 256)), exact integer exponents
  for (int e = tid; e < 256; e += kT) {
    float sn, cs;
    sincospif((float)((e >> 4) * (e & 15)) / 128.f, &sn, &cs);
    sm.tw[e >> 4][e & 15] = make_float2(cs, -sn);
  }
  const uint32_t polls = a.wait_polls ? a.wait_polls - 1 : kPolls;
  const uint32_t total = (uint32_t)fsch_total(a.sc);
  bool failed = false;
  // Thread kSched (lane 0 of warp 1) claims the next ticket when an item starts, and decodes it and
  // waits for its inputs when the item ends; thread 0 releases the finished item at the same time,
  // so the two round trips overlap. The smallest unfinished ticket is always some CTA's current
  // item (a CTA's claimed ticket is larger than its current one), and its inputs are complete, so
  // the grid progresses.
  constexpr int kSched = 32;
  uint32_t next = 0;
  if (tid == kSched) next = atomicAdd(a.ticket, 1u);
  for (int it = 0;; ++it) {
    if (tid == kSched) {
      const Work wk = take(a, next, total);
      const unsigned int *dep = wk.p >= 0 ? dep_of(a, wk) : nullptr;
      if (dep && !wait_count(dep, kJ, polls)) failed = true;
      work[it & 1] = wk;
    }
    __syncthreads();
    const Work wk = work[it & 1];
    if (wk.p < 0) break;
    if (tid == kSched) next = atomicAdd(a.ticket, 1u);
    if (wk.p & 1) row_item<Odd>(a, sm, wk, sm.d);
    else col_item(a, sm, wk, sm.d);
    __syncthreads();  // every thread's stores of the item precede the release below
    if (tid == 0)
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.done + wk.f * a.sc.P + wk.p) : "memory");
  }
  if (failed && a.status) *(volatile unsigned int *)a.status = 1u;
}

// The four-step twiddles of every launch: [0, N) holds W_N^(k1 b) at [k1][b] (k1, b < 256), and
// [N, 2N) the inverse, conj(W_N^(k1 b)) / N, so a half warp reads 16 consecutive values of one k1.
__global__ void fft_l2_twiddle_kernel(float2 *t) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint32_t)kN) return;
  const uint32_t e = ((i >> 8) * (i & 255)) & (kN - 1);
  float sn, cs;
  sincospif((float)e / (float)(kN / 2), &sn, &cs);
  t[i] = make_float2(cs, -sn);
  t[kN + i] = make_float2(cs * (1.f / kN), sn * (1.f / kN));
}

}  // namespace

size_t fft_l2_smem_bytes() { return sizeof(Smem); }

// Built once per device, on a private stream, and kept until the process exits (1 MB); the first
// call on a device allocates, so it cannot be part of a stream capture.
cudaError_t fft_l2_twiddles(const float2 **out) {
  static std::mutex mu;
  static float2 *tables[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!tables[dev]) {
    float2 *t = nullptr;
    e = cudaMalloc(&t, 2 * (size_t)kN * sizeof(float2));
    if (e != cudaSuccess) return e;
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      fft_l2_twiddle_kernel<<<kN / 256, 256, 0, st>>>(t);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    if (e != cudaSuccess) {
      cudaFree(t);
      return e;
    }
    tables[dev] = t;
  }
  *out = tables[dev];
  return cudaSuccess;
}

int fft_l2_ctas_per_sm() {
  static std::atomic<int> cached[64];
  static std::atomic<bool> init[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 0;
  }
  if (init[dev].load()) return cached[dev].load();
  int n = 0, n1 = 0;
  if (cudaFuncSetAttribute(fft_l2_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)) !=
          cudaSuccess ||
      cudaFuncSetAttribute(fft_l2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fft_l2_kernel<false>, kT, sizeof(Smem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, fft_l2_kernel<true>, kT, sizeof(Smem)) != cudaSuccess)
    n = n1 = 0;
  n = std::min(n, n1);  // both instantiations are sized by the same grid
  cudaGetLastError();
  cached[dev].store(n);
  init[dev].store(true);
  return n;
}

// Slices of G rows such that a phase's items are claimed kFftL2Items G L P tickets (about 2.5
// grids) after the items they read: each CTA holds its item and one claimed ticket, so up to two
// grids of tickets are claimed and unfinished at a time (1.25 grids measured 4 % slower at 256
// rows). The ring holds (P - 1) L + 3 slices, so a slot is refilled two steps after its last reader
// was claimed.
bool fft_l2_plan(int64_t nfft, int nsteps, int ctas, FftL2Plan *out) {
  if (nfft < 1 || nsteps < 1 || nsteps > kFftMaxSteps || ctas < 1) return false;
  FftSched c{};
  c.nfft = nfft;
  c.P = nsteps + 1;
  c.L = 2;
  const int64_t want = (5LL * ctas + 1) / 2;
  const int64_t per_slice_row = (int64_t)kFftL2Items * c.L * c.P;
  c.G = (int32_t)std::max<int64_t>(1, (want + per_slice_row - 1) / per_slice_row);
  c.nslices = (nfft + c.G - 1) / c.G;
  if (c.nslices < c.L) c.L = (int32_t)c.nslices;
  if (fsch_total(c) >= (1LL << 31)) return false;  // tickets are 32-bit
  out->sc = c;
  out->ring_rows = std::min<int64_t>(c.nslices, (int64_t)(c.P - 1) * c.L + 3) * c.G;
  out->ctas = (int)std::min<int64_t>(ctas, fsch_total(c));
  out->ring_bytes = (size_t)out->ring_rows * kN * sizeof(float2);
  out->counter_bytes = ((size_t)nfft * c.P + 1) * sizeof(unsigned int);
  return true;
}

int64_t fsch_total_tickets(const FftSched &c) { return fsch_total(c); }

// Every (phase, row, item) has exactly one ticket, and every wait of the kernel is on an item with
// a smaller ticket.
bool fft_l2_schedule_ok(const FftSched &c, int64_t ring_rows) {
  const int64_t total = fsch_total(c);
  if (fsch_pairs_before(c, fsch_steps(c)) * kFftL2Items * c.G != total) return false;
  std::vector<uint8_t> seen((size_t)total, 0);
  for (int64_t T = 0; T < total; ++T) {
    int p, j;
    int64_t f;
    fsch_decode(c, T, &p, &f, &j);
    int p2, j2;
    int64_t f2;
    fsch_decode32(c, (uint32_t)T, &p2, &f2, &j2);
    if (p2 != p || f2 != f || j2 != j) return false;
    if (p < 0 || p >= c.P || f < 0 || f >= c.nslices * c.G || j < 0 || j >= kFftL2Items) return false;
    if (fsch_ticket(c, p, f, j) != T) return false;
    uint8_t &s = seen[((size_t)f * c.P + p) * kFftL2Items + j];
    if (s) return false;
    s = 1;
    if (f >= c.nfft) continue;
    if (p > 0)
      for (int i = 0; i < kFftL2Items; ++i)
        if (fsch_ticket(c, p - 1, f, i) >= T) return false;
    if (p == 0 && f >= ring_rows)
      for (int i = 0; i < kFftL2Items; ++i)
        if (fsch_ticket(c, c.P - 1, f - ring_rows, i) >= T) return false;
  }
  return true;
}

cudaError_t launch_fft_l2(const FftL2Args &a, int ctas, cudaStream_t s) {
  if (a.nsteps < 1 || a.nsteps > kFftMaxSteps || a.sc.P != a.nsteps + 1 || a.sc.nfft < 1 || ctas < 1 ||
      a.ring_rows < 1 || !a.ring || !a.done || a.ticket != a.done + a.sc.nfft * a.sc.P)
    return cudaErrorInvalidValue;
  const bool odd = a.nsteps & 1;
  cudaError_t e = cudaFuncSetAttribute(odd ? (const void *)fft_l2_kernel<true> : (const void *)fft_l2_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e == cudaSuccess)
    e = cudaMemsetAsync(a.done, 0, ((size_t)a.sc.nfft * a.sc.P + 1) * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (odd) fft_l2_kernel<true><<<dim3(ctas), dim3(kT), sizeof(Smem), s>>>(a);
  else fft_l2_kernel<false><<<dim3(ctas), dim3(kT), sizeof(Smem), s>>>(a);
  return cudaGetLastError();
}

}  // namespace mrw
