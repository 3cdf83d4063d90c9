// Stencil groups and batched instances: a 5x5 box blur fused between a prefix and a suffix of
// pointwise stages, over tiles staged in shared memory by TMA.
//
// A Pipeline whose stages include a stencil cannot keep the whole intermediate in registers: the
// blur reads a 2-pixel halo around each output tile. Following the paper's locality-aware
// decomposition (Section 3.1) the tile of the blur's input (prefix applied, halo included) is
// computed once into shared memory from a TMA-loaded box of the source image; the blur reads it
// there and the suffix runs on the blur's output before the single HBM write.
//
// Batching: every (instance, plane, tile) is one work item of a global tile list; a persistent
// grid takes items from a device counter, so thousands of uneven instances (the Map skeleton over
// independent images) run in one launch. Each instance has its own 3-D tensor map {W, H, D}.
//
// TMA rules kept here: the box's x start is rounded down to a multiple of 16 bytes and the box is
// widened to cover the rounded start; loads may start at negative coordinates (zero fill), and
// the kernel never reads a filled position because it clamps to the image (edge replication).
//
// Waits: only thread 0 waits on a TMA mbarrier, for a bounded number of polls; if the bound is
// reached it records MRW status word 1 and the whole CTA leaves after a second bounded wait for
// its copies in flight.
#include <atomic>
#include <mutex>

#include "mrw_internal.h"
#include "pixel_ops.cuh"

namespace mrw {
namespace {

constexpr int kBlock = 256;
constexpr uint32_t kWaitPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait: true if the phase completed within `polls` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint32_t polls = kWaitPolls) {
  for (uint32_t i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Geometry of one work item.
struct Tile {
  int inst;     // instance index, -1 = no tile
  int z, y0, x0;
  int W, H, rows, cols;  // plane size, valid output rows/cols of this tile
  int r0;       // first blur-output (R) column the tile needs
  int bx, by;   // TMA box origin (bx multiple of 16)
};

__device__ __forceinline__ Tile locate(const StencilArgs &a, int64_t t) {
  Tile g;
  g.inst = -1;
  if (t >= a.total_tiles) return g;
  int lo = 0, hi = a.ninst - 1;  // last instance with prefix <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.tile_prefix[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const StencilInstance in = a.inst[lo];
  const int64_t lt = t - a.tile_prefix[lo];
  const int64_t per_plane = (int64_t)in.tiles_x * in.tiles_y;
  g.inst = lo;
  g.z = (int)(lt / per_plane);
  const int rem = (int)(lt % per_plane);
  const int ty = rem / in.tiles_x, tx = rem % in.tiles_x;
  g.W = in.W;
  g.H = in.H;
  g.y0 = ty * a.tile_h;
  g.x0 = tx * a.tile_w;
  g.rows = min(a.tile_h, in.H - g.y0);
  g.cols = min(a.tile_w, in.W - g.x0);
  const int x1 = g.x0 + g.cols;
  g.r0 = a.msuf ? in.W - x1 : g.x0;
  const int h = a.halo;
  const int in_lo = a.mpre ? in.W - (g.r0 + g.cols) - h : g.r0 - h;
  g.bx = in_lo & ~15;
  g.by = g.y0 - h;
  return g;
}

// ---- per-pixel ops (general paths: edge quads, suffixes, more than two noise stages) ----
__device__ __forceinline__ uint32_t apply_ops_px(const ChainOp *ops, int n, uint32_t p, int col, int W, uint32_t y,
                                                 uint32_t seed_xor) {
  for (int i = 0; i < n; ++i) {
    const int kind = ops[i].kind;
    if (kind == OP_SOLARISE) {
      p = p < 128u ? p : 255u - p;
    } else if (kind == OP_THRESH) {
      const uint32_t t = ops[i].t;
      p = (p >= (t & 0xFFu) ? 1u : 0u) + (p >= ((t >> 8) & 0xFFu) ? 1u : 0u);
    } else if (kind == OP_NOISE) {
      const uint32_t x = ops[i].flip ? (uint32_t)(W - 1 - col) : (uint32_t)col;
      const uint32_t h = fmix32(fmix32(fmix32(ops[i].seed ^ seed_xor) ^ x) ^ y);
      const int q = (int)p + (int)(h % 41u) - 20;
      p = (uint32_t)min(max(q, 0), 255);
    }
  }
  return p;
}

// Ops on the 4 pixels of a word whose columns are c0..c0+3 (clamped columns gc[k] for the hash);
// colpre[kn] holds the 4 column hashes of noise op kn (already split as c ^ (c >> 16)).
struct Cols4 {
  int c[4];
};

__device__ __forceinline__ uint32_t apply_ops_word(const ChainOp *ops, int n, uint32_t w, uint4 colpre0,
                                                   uint4 colpre1, uint32_t ypre, Cols4 gc, int W,
                                                   uint32_t seed_xor) {
  int kn = 0;
  for (int i = 0; i < n; ++i) {
    const int kind = ops[i].kind;
    if (kind == OP_SOLARISE) {
      w = solarise4(w);
    } else if (kind == OP_THRESH) {
      const uint32_t t = ops[i].t;
      const uint32_t t0 = (t & 0xFFu) * 0x01010101u, t1 = ((t >> 8) & 0xFFu) * 0x01010101u;
      w = (ge4(w, t0, t0 & 0x7F7F7F7Fu) >> 7) + (ge4(w, t1, t1 & 0x7F7F7F7Fu) >> 7);
    } else if (kind == OP_NOISE) {
      uint32_t c[4];
      if (kn < kMaxNoisePerGroup) {
        const uint4 v = kn == 0 ? colpre0 : colpre1;
        c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t x = ops[i].flip ? (uint32_t)(W - 1 - gc.c[k]) : (uint32_t)gc.c[k];
          const uint32_t cc = fmix32(fmix32(ops[i].seed ^ seed_xor) ^ x);
          c[k] = cc ^ (cc >> 16);
        }
      }
      w = noise4(w, c[0], c[1], c[2], c[3], ypre);
      ++kn;
    }
  }
  return w;
}

// 4 bytes of a shared-memory row starting at byte offset o (o >= 0, any alignment; the row is
// 4-byte aligned and holds at least o + 4 bytes).
__device__ __forceinline__ uint32_t load4(const uint8_t *row, int o) {
  const uint32_t *r32 = reinterpret_cast<const uint32_t *>(row);
  const uint32_t lo = r32[o >> 2];
  if ((o & 3) == 0) return lo;
  const uint32_t hi = r32[(o >> 2) + 1];
  return __funnelshift_r(lo, hi, 8 * (o & 3));
}

// Store the first nb (1..4) bytes of w at p (p 4-byte aligned when nb == 4).
__device__ __forceinline__ void store4(uint8_t *p, uint32_t w, int nb) {
  if (nb >= 4) {
    *reinterpret_cast<uint32_t *>(p) = w;
  } else {
    for (int k = 0; k < nb; ++k) p[k] = (uint8_t)(w >> (8 * k));
  }
}

template <int TW, int H>
__global__ void __launch_bounds__(kBlock) stencil_kernel(const __grid_constant__ StencilArgs a) {
  constexpr int QP = (TW + 2 * H + 15) & ~15;  // Q row pitch (bytes) and column-hash row length
  constexpr int QW4 = (TW + 2 * H + 3) / 4;    // quads per Q row
  constexpr int RQ = TW / 4;                   // quads per output row
  constexpr int RPT = 4;                       // output rows per blur task
  extern __shared__ __align__(128) uint8_t smem[];
  const int BW = a.box_w, BH = a.box_h, TH = a.tile_h;
  // two TMA destination buffers: buffer b starts at smem + b * BH * BW
  uint8_t *qt = smem + 2 * BH * BW;
  uint8_t *rt = qt + BH * QP;
  uint32_t *qcol = reinterpret_cast<uint32_t *>(rt + TH * TW);  // [kMaxNoisePerGroup][QP]
  uint64_t *bar = reinterpret_cast<uint64_t *>(qcol + kMaxNoisePerGroup * QP);
  __shared__ int64_t s_tile[2];
  __shared__ Tile s_geo[2];  // geometry of the tile in each buffer, computed once by thread 0
  __shared__ int s_fail;

  const int tid = threadIdx.x;
  const uint32_t box_bytes = (uint32_t)(BW * BH);
  uint32_t phases = 0u;  // bit b = parity of buffer b's next completion
  // no suffix: the last phase writes the output straight from registers
  const bool direct = a.nsuf == 0 && a.msuf == 0;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    const int64_t t = atomicAdd(a.queue, 1u);
    s_tile[0] = t;
    if (t < a.total_tiles) {
      const Tile g = locate(a, t);
      s_geo[0] = g;
      mbar_expect_tx(&bar[0], box_bytes);
      tma_load_3d(smem, a.maps + g.inst, g.bx, g.by, g.z, &bar[0]);
    }
  }
  __syncthreads();

  int cur = 0;
  while (true) {
    const int64_t t = s_tile[cur];
    if (t >= a.total_tiles) break;
    const Tile g = s_geo[cur];
    const int64_t out_off = a.inst[g.inst].out_off;
    const int32_t pitch_out = a.inst[g.inst].pitch_out;
    const uint32_t seed_xor = a.inst[g.inst].seed_xor;

    // Prefetch the next tile into the other buffer (free since the end of the previous iteration).
    if (tid == 0) {
      const int64_t tn = atomicAdd(a.queue, 1u);
      s_tile[cur ^ 1] = tn;
      if (tn < a.total_tiles) {
        const Tile gn = locate(a, tn);
        s_geo[cur ^ 1] = gn;
        fence_proxy_async();
        mbar_expect_tx(&bar[cur ^ 1], box_bytes);
        tma_load_3d(smem + (cur ^ 1) * BH * BW, a.maps + gn.inst, gn.bx, gn.by, gn.z, &bar[cur ^ 1]);
      }
      if (!mbar_wait_bounded(&bar[cur], (phases >> cur) & 1u, a.wait_polls ? a.wait_polls - 1 : kWaitPolls))
        s_fail = 1;
    }
    // Column hashes of the prefix's noise ops for this tile's Q columns: c ^ (c >> 16) with
    // c = F(F(seed ^ instance seed) ^ x), x the op's column coordinate of the clamped Q column.
    const int qcols = g.cols + 2 * H;
    {
      int kn = 0;
      for (int i = 0; i < a.npre && kn < kMaxNoisePerGroup; ++i) {
        if (a.pre[i].kind != OP_NOISE) continue;
        const uint32_t fs = fmix32(a.pre[i].seed ^ seed_xor);
        const int flip = a.pre[i].flip;
        for (int j = tid; j < 4 * QW4; j += kBlock) {
          const int gc = min(max(g.r0 - H + j, 0), g.W - 1);
          const uint32_t x = flip ? (uint32_t)(g.W - 1 - gc) : (uint32_t)gc;
          const uint32_t c = fmix32(fs ^ x);
          qcol[kn * QP + j] = c ^ (c >> 16);
        }
        ++kn;
      }
    }
    __syncthreads();
    if (s_fail) break;
    phases ^= 1u << cur;

    const uint8_t *bx = smem + cur * BH * BW;
    const uint32_t plane_row0 = (uint32_t)g.z * (uint32_t)g.H;
    uint8_t *obase = a.out_base + out_off + ((int64_t)g.z * g.H + g.y0) * pitch_out + g.x0;

    // Phase A: Q words (prefix applied to the clamped neighbourhood), 4 columns per task.
    const int qrows = g.rows + 2 * H;
    const int nq4 = (qcols + 3) >> 2;
    for (int e = tid; e < qrows * QW4; e += kBlock) {
      const int i = e / QW4, jq = e - i * QW4;
      if (jq >= nq4) continue;
      const int gy = min(max(g.y0 - H + i, 0), g.H - 1);
      const uint8_t *brow = bx + (gy - g.by) * BW;
      const int c0 = g.r0 - H + 4 * jq;
      Cols4 gc;  // clamped (edge-replicated) columns of the quad
      uint32_t w;
      if (c0 >= 0 && c0 + 3 <= g.W - 1 && 4 * jq + 4 <= qcols) {
#pragma unroll
        for (int k = 0; k < 4; ++k) gc.c[k] = c0 + k;
        // a whole quad inside the image and inside the tile's Q range: one (funnel-shifted) word
        if (!a.mpre) {
          w = load4(brow, c0 - g.bx);
        } else {
          w = __byte_perm(load4(brow, g.W - 4 - c0 - g.bx), 0, 0x0123);
        }
      } else {
        // image edges (replicated columns) and the tile's ragged last quad
        w = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) gc.c[k] = min(max(c0 + k, 0), g.W - 1);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (4 * jq + k < qcols) {
            const int ic = a.mpre ? g.W - 1 - gc.c[k] : gc.c[k];
            w |= (uint32_t)brow[ic - g.bx] << (8 * k);
          }
        }
      }
      const uint32_t y = plane_row0 + (uint32_t)gy;
      const uint4 cp0 = *reinterpret_cast<const uint4 *>(qcol + 4 * jq);
      const uint4 cp1 = *reinterpret_cast<const uint4 *>(qcol + QP + 4 * jq);
      w = apply_ops_word(a.pre, a.npre, w, cp0, cp1, y ^ (y >> 16), gc, g.W, seed_xor);
      if (H == 0 && direct) {
        store4(obase + (int64_t)i * pitch_out + 4 * jq, w, min(4, g.cols - 4 * jq));
      } else {
        *reinterpret_cast<uint32_t *>(qt + i * QP + 4 * jq) = w;
      }
    }
    if (!(H == 0 && direct)) {
      __syncthreads();
      const uint8_t *rsrc = qt;  // R tile: the blur output, or Q itself without a blur
      int rpitch = QP;
      if (H == 2) {
        // Phase B: 5x5 box sums. A task is 4 output columns x RPT rows: horizontal 5-sums of each
        // Q row in packed 16-bit lanes (h0,h2) and (h1,h3), vertical sums over a sliding window.
        const int nr4 = (g.cols + 3) >> 2;
        const int ntask = ((g.rows + RPT - 1) / RPT) * RQ;
        for (int e = tid; e < ntask; e += kBlock) {
          const int rg = e / RQ, jr = e - rg * RQ;
          if (jr >= nr4) continue;
          const int i0 = rg * RPT, ni = min(RPT, g.rows - i0);
          uint32_t h02[RPT + 4], h13[RPT + 4];
          uint32_t s02 = 0, s13 = 0;
#pragma unroll
          for (int d = 0; d < RPT + 4; ++d) {
            if (d < ni + 4) {
              const uint32_t *qw = reinterpret_cast<const uint32_t *>(qt + (i0 + d) * QP + 4 * jr);
              const uint32_t lo = qw[0], hi = qw[1];
              const uint32_t E = lo & 0x00FF00FFu, O = (lo >> 8) & 0x00FF00FFu;
              const uint32_t E2 = hi & 0x00FF00FFu, O2 = (hi >> 8) & 0x00FF00FFu;
              const uint32_t A = E + O, A2 = E2 + O2, P = __byte_perm(A, A2, 0x5432);
              h02[d] = A + P + E2;
              h13[d] = O + P + A2;
              s02 += h02[d];
              s13 += h13[d];
              if (d >= 5) {
                s02 -= h02[d - 5];
                s13 -= h13[d - 5];
              }
              if (d >= 4) {
                const int r = i0 + d - 4;
                const uint32_t o = ((s02 & 0xFFFFu) + 12u) / 25u | ((((s13 & 0xFFFFu) + 12u) / 25u) << 8) |
                                   ((((s02 >> 16) + 12u) / 25u) << 16) | ((((s13 >> 16) + 12u) / 25u) << 24);
                if (direct) {
                  store4(obase + (int64_t)r * pitch_out + 4 * jr, o, min(4, g.cols - 4 * jr));
                } else {
                  *reinterpret_cast<uint32_t *>(rt + r * TW + 4 * jr) = o;
                }
              }
            }
          }
        }
        rsrc = rt;
        rpitch = TW;
        if (!direct) __syncthreads();
      }
      if (!direct) {
        // Suffix and store (general path): one 16-byte output segment per thread and row.
        const int segs = (g.cols + 15) >> 4;
        for (int e = tid; e < segs * g.rows; e += kBlock) {
          const int i = e / segs, c = e - i * segs;
          const int nv = min(16, g.cols - 16 * c);
          const uint8_t *rrow = rsrc + i * rpitch;
          const uint32_t y = plane_row0 + (uint32_t)(g.y0 + i);
          uint8_t *orow = obase + (int64_t)i * pitch_out + 16 * c;
          for (int k = 0; k < nv; ++k) {
            const int lc = a.msuf ? g.cols - 1 - 16 * c - k : 16 * c + k;
            orow[k] = (uint8_t)apply_ops_px(a.suf, a.nsuf, rrow[lc], g.x0 + 16 * c + k, g.W, y, seed_xor);
          }
        }
      }
    }
    __syncthreads();
    cur ^= 1;
  }

  if (s_fail && tid == 0) {
    *(volatile unsigned int *)a.status = 1u;  // may be mapped host memory
    // let the copies this CTA issued land before it leaves (bounded as well)
    if (s_tile[cur ^ 1] < a.total_tiles) (void)mbar_wait_bounded(&bar[cur ^ 1], (phases >> (cur ^ 1)) & 1u);
    (void)mbar_wait_bounded(&bar[cur], (phases >> cur) & 1u);
  }
}

// ---- Row-streaming blur kernel --------------------------------------------------------------
//
// Groups of the form (pointwise prefix, 5x5 blur) with at most kMaxNoisePerGroup noise stages
// and no suffix — the batched Filter Pipeline + blur among them — run here instead of through
// the 2-D tile kernel above. Each warp is an independent worker:
//   * a work item is a strip of kRowsStrip (124) output columns by tile_h rows of one plane;
//     lane l owns the 4 blur-input (Q) columns x0 - 2 + 4l .. x0 + 1 + 4l and, for l < 31, the 4
//     output columns x0 + 4l .. x0 + 3 + 4l;
//   * the warp streams the item's source rows through a ring of kRowsBufs TMA boxes of
//     kRowsBoxW x kRowsChunk bytes in its own slice of shared memory, issued ahead by lane 0;
//   * per source row, each lane applies the prefix to its 4 pixels in registers, takes the two
//     Q columns right of its quad from lane l + 1 (one shuffle) and forms the horizontal 5-sums of
//     its 4 output columns in packed 16-bit lanes; a 5-row window of those sums in registers gives
//     the vertical sums, so every source row is read and transformed once per item;
//   * edge replication: a lane whose quad crosses the image's left or right edge reads clamped
//     columns; rows above the image repeat the first row's sums and rows below repeat the last's.
// Items are claimed from the global tile counter; within an instance the strips of one row band
// are consecutive, so neighbouring strips write their shared 32-byte sectors at about the same
// time.
constexpr int kRowsBufs = 4;
constexpr int kRowsFifo = kRowsBufs + 2;
constexpr int kRowsWarps = 8;
constexpr int kRowsBlock = 32 * kRowsWarps;
constexpr uint32_t kRowsBoxBytes = (uint32_t)(kRowsBoxW * kRowsChunk);

// A work item, decoded by the warp's issuer and read by its consumer.
struct RowItem {
  int64_t out_off;
  int32_t inst, z, x0, ys, ye, W, H, pitch_out;
  int32_t qa;       // image row of the first box row: ys - 2 (may be negative)
  int32_t nchunks;  // boxes of kRowsChunk rows covering rows ys - 2 .. ye + 1
  int32_t bx;       // box column origin (multiple of 16)
  uint32_t seed_xor;
};

// Issue-side state of a warp: every lane holds the same copy in registers (the lanes run the
// issue path together; lane 0 alone writes shared memory and starts the copies). The item being
// issued is in FIFO slot (tail - 1) % kRowsFifo.
struct RowIssue {
  int32_t j;        // next chunk of the item being issued
  int32_t nchunks;  // chunks of that item (-1: the tile counter is exhausted)
  int32_t count;    // chunks issued so far
  int32_t tail;     // FIFO slots written so far
};

struct alignas(128) RowWarpSmem {
  uint8_t buf[kRowsBufs][kRowsChunk][kRowsBoxW];
  // column halves of each noise op's hashes for lane l's 4 Q columns (written and read by lane l
  // only; kept here rather than in registers, which the row loop needs)
  uint4 cp[kMaxNoisePerGroup][32];
  uint64_t bar[kRowsBufs];
  RowItem fifo[kRowsFifo];
};

// Index of the last instance whose first tile is <= t (all lanes; ninst >= 1). Each round the 32
// lanes probe evenly spaced prefix entries of the remaining range and a ballot keeps one stride.
__device__ __forceinline__ int warp_find_instance(const int64_t *prefix, int ninst, int64_t t, int lane) {
  int lo = 0, hi = ninst;  // prefix[lo] <= t < prefix[hi]
  while (hi - lo > 1) {
    const int span = hi - lo;
    const int step = (span + 31) >> 5;
    const int idx = lo + lane * step;
    const bool le = idx < hi && __ldg(prefix + idx) <= t;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, le);
    const int k = 31 - __clz((int)m);  // lane 0 always qualifies
    lo = lo + k * step;
    hi = min(lo + step, hi);
  }
  return lo;
}

// Claims the next work item from the tile counter and decodes it into FIFO slot `slot` (all lanes
// call it; lane 0 writes the slot). Returns the item's chunk count, or -1 when the counter is
// exhausted (the slot then holds the end marker). The issue state stays in the caller's registers:
// a reference to it here would put it in local memory.
template <bool MIR>
__device__ __noinline__ int rows_claim(const StencilArgs &a, RowWarpSmem &w, int slot, int lane) {
  unsigned int t = 0;
  if (lane == 0) t = atomicAdd(a.queue, 1u);
  t = __shfl_sync(0xFFFFFFFFu, t, 0);
  RowItem it;
  if ((int64_t)t >= a.total_tiles) {
    it.inst = -1;
    it.nchunks = -1;
  } else {
    const int i = warp_find_instance(a.tile_prefix, a.ninst, (int64_t)t, lane);
    const StencilInstance in = a.inst[i];
    // tile index within the instance and tiles per plane both fit 32 bits
    const int lt = (int)((int64_t)t - a.tile_prefix[i]);
    const int per_plane = in.tiles_x * in.tiles_y;
    const int z = lt / per_plane;
    const int rem = lt - z * per_plane;
    const int seg = rem / in.tiles_x, strip = rem - seg * in.tiles_x;
    it.inst = i;
    it.z = z;
    it.x0 = strip * kRowsStrip;
    it.ys = seg * a.tile_h;
    it.ye = min(it.ys + a.tile_h, in.H);
    it.W = in.W;
    it.H = in.H;
    it.pitch_out = in.pitch_out;
    it.out_off = in.out_off;
    it.seed_xor = in.seed_xor;
    it.qa = it.ys - 2;  // box row 0 = image row ys - 2 (negative rows read the fill value)
    it.nchunks = (it.ye - it.ys + 4 + kRowsChunk - 1) / kRowsChunk;
    it.bx = MIR ? ((in.W - it.x0 - 126) & ~15) : ((it.x0 - 2) & ~15);
  }
  if (lane == 0) w.fifo[slot] = it;
  __syncwarp();
  return it.nchunks;
}

// Starts the copy of one more chunk into the ring, claiming a new item when the current one is
// fully issued (all lanes call it).
template <bool MIR>
__device__ __forceinline__ void rows_issue(const StencilArgs &a, RowWarpSmem &w, RowIssue &st, int lane) {
  if (st.nchunks < 0) return;
  if (st.j == st.nchunks) {  // the item is fully issued (or none was claimed yet)
    st.nchunks = rows_claim<MIR>(a, w, st.tail % kRowsFifo, lane);
    st.tail += 1;
    st.j = 0;
    if (st.nchunks < 0) return;
  }
  if (lane == 0) {
    const RowItem &it = w.fifo[(st.tail - 1) % kRowsFifo];
    const int b = st.count % kRowsBufs;
    fence_proxy_async();
    mbar_expect_tx(&w.bar[b], kRowsBoxBytes);
    tma_load_3d(&w.buf[b][0][0], a.maps + it.inst, it.bx, it.qa + st.j * kRowsChunk, it.z, &w.bar[b]);
  }
  st.j += 1;
  st.count += 1;
}

// Bounded wait of the whole warp on chunk s's barrier; the result is the same on every lane.
__device__ __forceinline__ bool rows_wait(RowWarpSmem &w, int s, uint32_t polls) {
  const bool ok = mbar_wait_bounded(&w.bar[s % kRowsBufs], (uint32_t)(s / kRowsBufs) & 1u, polls);
  return __all_sync(0xFFFFFFFFu, ok);
}

// Per-lane state of the item being consumed: only what the row loop needs stays in registers.
struct RowLane {
  uint8_t *orow;     // this lane's output quad in the next output row
  int32_t pitch_out;
  int32_t wi;        // first of the two 32-bit words of a box row that hold the lane's 4 Q pixels
  uint32_t sel;      // byte_perm selector picking the 4 Q pixels out of those 8 bytes (reversed
                     // for a mirrored prefix, edge columns replicated)
  int32_t nout;      // output bytes of the lane's quad (0: none)
  uint32_t yrow;     // global row (plane * H + row) of the item's first source row, for the hash
};

// The lane's 4 Q pixels of one box row (Q column c0 + k in byte k).
__device__ __forceinline__ uint32_t rows_quad(const uint8_t *row, const RowLane &L) {
  const uint32_t *r32 = reinterpret_cast<const uint32_t *>(row) + L.wi;
  return __byte_perm(r32[0], r32[1], L.sel);
}

// Prefix ops on the lane's quads of G consecutive source rows (row j's hash row is y0 + j): each
// op is decoded once for the G rows, whose 4 G pixels are independent work for the scheduler.
template <int NN, int G>
__device__ __forceinline__ void rows_prefix_g(const StencilArgs &a, uint32_t (&q)[G], const uint4 *cp, uint32_t y0) {
  uint32_t yp[G];
#pragma unroll
  for (int j = 0; j < G; ++j) {
    const uint32_t y = y0 + (uint32_t)j;
    yp[j] = y ^ (y >> 16);
  }
  // common sequences first: one uniform branch instead of a walk over the op list
  const int pat = a.pre_pattern;
  if (pat == PAT_NONE) return;
  if (pat == PAT_SOLARISE) {
#pragma unroll
    for (int j = 0; j < G; ++j) q[j] = solarise4(q[j]);
    return;
  }
  if constexpr (NN >= 1) {
    if (pat == PAT_NOISE || pat == PAT_NOISE_SOLARISE) {
      const uint4 c = cp[0];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        q[j] = noise4(q[j], c.x, c.y, c.z, c.w, yp[j]);
        if (pat == PAT_NOISE_SOLARISE) q[j] = solarise4(q[j]);
      }
      return;
    }
  }
  int kn = 0;
  for (int i = 0; i < a.npre; ++i) {
    const int kind = a.pre[i].kind;
    if (kind == OP_SOLARISE) {
#pragma unroll
      for (int j = 0; j < G; ++j) q[j] = solarise4(q[j]);
    } else if (kind == OP_THRESH) {
      const uint32_t t = a.pre[i].t;
      const uint32_t t0 = (t & 0xFFu) * 0x01010101u, t1 = ((t >> 8) & 0xFFu) * 0x01010101u;
#pragma unroll
      for (int j = 0; j < G; ++j)
        q[j] = (ge4(q[j], t0, t0 & 0x7F7F7F7Fu) >> 7) + (ge4(q[j], t1, t1 & 0x7F7F7F7Fu) >> 7);
    } else if (kind == OP_NOISE) {
      if constexpr (NN >= 1) {
        if (kn < NN) {
          const uint4 c = cp[kn * 32];
#pragma unroll
          for (int j = 0; j < G; ++j) q[j] = noise4(q[j], c.x, c.y, c.z, c.w, yp[j]);
        }
      }
      ++kn;
    }
  }
}

// Rows of source data a lane transforms together (two groups per TMA box).
constexpr int kRowsGroup = 4;
static_assert(kRowsChunk % kRowsGroup == 0, "a row group must not straddle two boxes");

// MINB: CTAs per SM the registers are budgeted for (4: 64 registers; 3: 80).
template <int NN, bool MIR, int MINB>
__global__ void __launch_bounds__(kRowsBlock, MINB) stencil_rows_kernel(const __grid_constant__ StencilArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  RowWarpSmem &w = reinterpret_cast<RowWarpSmem *>(smem)[threadIdx.x >> 5];

  if (lane == 0) {
    for (int b = 0; b < kRowsBufs; ++b) mbar_init(&w.bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  RowIssue st{};  // j == nchunks == 0: the first call claims an item
  for (int k = 0; k < kRowsBufs; ++k) rows_issue<MIR>(a, w, st, lane);

  int cur = 0;   // boxes consumed so far
  int head = 0;  // FIFO slots consumed so far
  bool failed = false;
  while (true) {
    const RowItem &it = w.fifo[head % kRowsFifo];
    ++head;
    if (it.inst < 0) break;
    RowLane L;
    {
      const int W = it.W;
      const int c0 = it.x0 - 2 + 4 * lane;
      // column halves of the noise hashes of this lane's (clamped) Q columns
      if constexpr (NN > 0) {
        int kn = 0;
        for (int i = 0; i < a.npre && kn < NN; ++i) {
          if (a.pre[i].kind != OP_NOISE) continue;
          const uint32_t fs = fmix32(a.pre[i].seed ^ it.seed_xor);
          const int flip = a.pre[i].flip;
          uint32_t v[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int cc = min(max(c0 + k, 0), W - 1);
            const uint32_t c = fmix32(fs ^ (uint32_t)(flip ? W - 1 - cc : cc));
            v[k] = c ^ (c >> 16);
          }
          w.cp[kn][lane] = make_uint4(v[0], v[1], v[2], v[3]);
          ++kn;
        }
      }
      // box offsets of the 4 (clamped, possibly mirrored) source columns; they span at most 4
      // consecutive bytes, which lie in the two words from word `wi` on
      int off[4], lo = 1 << 30;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int cc = min(max(c0 + k, 0), W - 1);
        off[k] = (MIR ? W - 1 - cc : cc) - it.bx;
        lo = min(lo, off[k]);
      }
      L.wi = lo >> 2;
      L.sel = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) L.sel |= (uint32_t)(off[k] - 4 * L.wi) << (4 * k);
      const int xo = it.x0 + 4 * lane;
      L.nout = lane < 31 ? max(0, min(4, W - xo)) : 0;
      L.pitch_out = it.pitch_out;
      L.orow = a.out_base + it.out_off + ((int64_t)it.z * it.H + it.ys) * it.pitch_out + xo;
      L.yrow = (uint32_t)it.z * (uint32_t)it.H + (uint32_t)it.qa;
    }
    // Virtual row v = box row v = image row ys - 2 + v, for v < nv. Rows above the image take
    // row 0's horizontal sums (virtual row vtop), rows below it row H - 1's (virtual row vbot).
    const int nv = it.ye - it.ys + 4;
    const int vtop = 2 - it.ys, vbot = it.H + 1 - it.ys;
    // Output row ys + 4k - 4 + j is the 5-row sum of virtual rows 4k - 4 + j .. 4k + j: the suffix
    // sums of group k - 1 plus the prefix sums of group k, in packed 16-bit lanes (+12: round half up).
    uint32_t p02[kRowsGroup] = {0, 0, 0, 0}, p13[kRowsGroup] = {0, 0, 0, 0};
    for (int k = 0; 4 * k < nv; ++k) {
      if (k > 0 && (k % (kRowsChunk / kRowsGroup)) == 0) {
        __syncwarp();
        ++cur;
        rows_issue<MIR>(a, w, st, lane);
      }
      if (k % (kRowsChunk / kRowsGroup) == 0 && !rows_wait(w, cur, a.wait_polls ? a.wait_polls - 1 : kWaitPolls)) {
        failed = true;
        break;
      }
      const uint8_t *box = &w.buf[cur % kRowsBufs][(4 * k) % kRowsChunk][0];
      uint32_t q[kRowsGroup];
#pragma unroll
      for (int j = 0; j < kRowsGroup; ++j) q[j] = rows_quad(box + j * kRowsBoxW, L);
      rows_prefix_g<NN, kRowsGroup>(a, q, &w.cp[0][lane], L.yrow + (uint32_t)(4 * k));
      uint32_t h02[kRowsGroup], h13[kRowsGroup];
#pragma unroll
      for (int j = 0; j < kRowsGroup; ++j) {
        // horizontal 5-sums of output columns 0..3 (Q bytes k .. k + 4 of this lane's quad and
        // the next lane's), packed as (0, 2) and (1, 3) in 16-bit lanes; the next lane's even
        // bytes E2 and pair sums A2 come from it by shuffle, already unpacked
        const uint32_t E = __byte_perm(q[j], 0, 0x4240), O = __byte_perm(q[j], 0, 0x4341);
        const uint32_t A = E + O;
        const uint32_t E2 = __shfl_down_sync(0xFFFFFFFFu, E, 1), A2 = __shfl_down_sync(0xFFFFFFFFu, A, 1);
        const uint32_t P = __byte_perm(A, A2, 0x5432);
        h02[j] = A + P + E2;
        h13[j] = O + P + A2;
      }
      if (k == 0 && vtop > 0) {  // rows above the image repeat row 0 (virtual row vtop <= 2)
#pragma unroll
        for (int j = 0; j < kRowsGroup - 1; ++j)
          if (j < vtop) {
            h02[j] = vtop == 1 ? h02[1] : h02[2];
            h13[j] = vtop == 1 ? h13[1] : h13[2];
          }
      }
      if (4 * k + kRowsGroup - 1 > vbot) {  // rows below the image repeat row H - 1
#pragma unroll
        for (int j = 0; j < kRowsGroup; ++j)
          if (4 * k + j > vbot) {
            h02[j] = j > 0 ? h02[j - 1] : p02[kRowsGroup - 1];
            h13[j] = j > 0 ? h13[j - 1] : p13[kRowsGroup - 1];
          }
      }
      if (k > 0) {
        uint32_t o[kRowsGroup];
        // the first output row's window is rows 4k - 4 .. 4k (+12 rounds half up); each next row
        // adds the entering row and drops the leaving one
        uint32_t v02 = (p02[0] + p02[1] + p02[2]) + (p02[3] + h02[0] + 0x000C000Cu);
        uint32_t v13 = (p13[0] + p13[1] + p13[2]) + (p13[3] + h13[0] + 0x000C000Cu);
#pragma unroll
        for (int j = 0; j < kRowsGroup; ++j) {
          if (j > 0) {
            v02 += h02[j] - p02[j - 1];
            v13 += h13[j] - p13[j - 1];
          }
          // x / 25 for x <= 25 * 255 + 12 in either 16-bit lane, as a multiplication (division by
          // an invariant integer, Granlund and Montgomery 1994): high lane mulhi(v, 5243) >> 1,
          // low lane the same on v << 16; 5243 = ceil(2^17 / 25), exact over the whole range of
          // both lanes whatever the other lane holds (checked exhaustively)
          const uint32_t d0 = __umulhi(v02 * 0x10000u, 5243u) >> 1, d2 = __umulhi(v02, 5243u) >> 1;
          const uint32_t d1 = __umulhi(v13 * 0x10000u, 5243u) >> 1, d3 = __umulhi(v13, 5243u) >> 1;
          o[j] = d0 + d1 * 0x100u + d2 * 0x10000u + d3 * 0x1000000u;
        }
        const int nrow = min(kRowsGroup, nv - 4 * k);  // output rows of this group (1..4)
        if (nrow == kRowsGroup && L.nout == 4) {
#pragma unroll
          for (int j = 0; j < kRowsGroup; ++j) *reinterpret_cast<uint32_t *>(L.orow + j * L.pitch_out) = o[j];
        } else if (L.nout > 0) {
#pragma unroll
          for (int j = 0; j < kRowsGroup; ++j)
            if (j < nrow) store4(L.orow + j * L.pitch_out, o[j], L.nout);
        }
        L.orow += kRowsGroup * L.pitch_out;
      }
#pragma unroll
      for (int j = 0; j < kRowsGroup; ++j) {
        p02[j] = h02[j];
        p13[j] = h13[j];
      }
    }
    if (failed) break;
    __syncwarp();
    ++cur;
    rows_issue<MIR>(a, w, st, lane);
  }

  if (failed) {
    if (lane == 0) {
      *(volatile unsigned int *)a.status = 1u;  // may be mapped host memory
      // let this warp's copies in flight land before it leaves (bounded as well)
      const int issued = st.count;
      for (int s = cur; s < issued; ++s)
        (void)mbar_wait_bounded(&w.bar[s % kRowsBufs], (uint32_t)(s / kRowsBufs) & 1u);
    }
    __syncwarp();
  }
}

const void *stencil_fn(int tile_w, int halo) {
  if (halo == 2) {
    switch (tile_w) {
      case 64: return (const void *)stencil_kernel<64, 2>;
      case 224: return (const void *)stencil_kernel<224, 2>;
      default: return (const void *)stencil_kernel<128, 2>;
    }
  }
  switch (tile_w) {
    case 64: return (const void *)stencil_kernel<64, 0>;
    case 224: return (const void *)stencil_kernel<224, 0>;
    default: return (const void *)stencil_kernel<128, 0>;
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

int stencil_tile_width(int requested) {
  return requested <= 64 ? 64 : (requested <= 128 ? 128 : 224);
}

size_t stencil_smem_bytes(int tile_h, int tile_w, int halo) {
  const int BW = (tile_w + 2 * halo + 15 + 15) & ~15;
  const int BH = tile_h + 2 * halo;
  const int QP = (tile_w + 2 * halo + 15) & ~15;
  size_t b = (size_t)2 * BH * BW + (size_t)BH * QP + (size_t)tile_h * tile_w;
  b += (size_t)4 * kMaxNoisePerGroup * QP;
  b = (b + 7) & ~(size_t)7;
  return b + 2 * sizeof(uint64_t);
}

namespace {
template <int MINB>
const void *stencil_rows_fn_b(int n_noise, int mirror) {
  switch (n_noise * 2 + (mirror ? 1 : 0)) {
    case 0: return (const void *)stencil_rows_kernel<0, false, MINB>;
    case 1: return (const void *)stencil_rows_kernel<0, true, MINB>;
    case 2: return (const void *)stencil_rows_kernel<1, false, MINB>;
    case 3: return (const void *)stencil_rows_kernel<1, true, MINB>;
    case 4: return (const void *)stencil_rows_kernel<2, false, MINB>;
    case 5: return (const void *)stencil_rows_kernel<2, true, MINB>;
    default: return nullptr;
  }
}

// The variant budgeted for 4 CTAs per SM serves requests of 4 or more, the other fewer.
const void *stencil_rows_fn(int n_noise, int mirror, int cps) {
  return cps >= 4 ? stencil_rows_fn_b<4>(n_noise, mirror) : stencil_rows_fn_b<3>(n_noise, mirror);
}

int count_noise_ops(const ChainOp *ops, int n) {
  int c = 0;
  for (int i = 0; i < n; ++i) c += ops[i].kind == OP_NOISE;
  return c;
}
}  // namespace

size_t stencil_rows_smem_bytes() { return sizeof(RowWarpSmem) * kRowsWarps; }
int stencil_rows_block() { return kRowsBlock; }

// The kernels' shared-memory limits are attributes of each device's copy of the functions: set
// them once per device, under a lock, before the first launch on that device.
cudaError_t stencil_prepare() {
  static std::atomic<bool> done[256];
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  for (int h : {0, 2})
    for (int w : {64, 128, 224}) {
      e = cudaFuncSetAttribute(stencil_fn(w, h), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) return e;
    }
  for (int v = 0; v < 12; ++v) {
    e = cudaFuncSetAttribute(stencil_rows_fn((v >> 1) % 3, v & 1, v < 6 ? 4 : 3),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stencil_rows_smem_bytes());
    if (e != cudaSuccess) return e;
  }
  done[dev].store(true, std::memory_order_release);
  return cudaSuccess;
}

int stencil_rows_blocks_per_sm(int n_noise, int mirror, int cps) {
  static std::atomic<int> cache[3][2][2];
  if (n_noise < 0 || n_noise > 2) return 1;
  std::atomic<int> &c = cache[n_noise][mirror ? 1 : 0][cps >= 4 ? 1 : 0];
  const int known = c.load(std::memory_order_relaxed);
  if (known) return known;
  int nb = 0;
  if (stencil_prepare() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stencil_rows_fn(n_noise, mirror, cps), kRowsBlock,
                                                    stencil_rows_smem_bytes()) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  c.store(nb > 0 ? nb : 1, std::memory_order_relaxed);
  return nb > 0 ? nb : 1;
}

// The kernel of a stencil launch and its final arguments (the prefix's op pattern filled in);
// nullptr if the launch shape does not match the kernel it selects.
static const void *stencil_launch_fn(StencilArgs &a, int block, size_t smem) {
  a.pre_pattern = op_pattern(a.pre, a.npre, &a.pre_pattern_t);
  if (a.rows_kernel) {
    const int nn = count_noise_ops(a.pre, a.npre);
    if (!stencil_rows_eligible(a.halo, a.nsuf, a.msuf, nn) || block != kRowsBlock ||
        smem != stencil_rows_smem_bytes() || a.tile_w != kRowsStrip || a.box_w != kRowsBoxW ||
        a.box_h != kRowsChunk || a.tile_h < 1)
      return nullptr;
    return stencil_rows_fn(nn, a.mpre, a.rows_cps);
  }
  if (block != kBlock || smem > 200 * 1024 || stencil_tile_width(a.tile_w) != a.tile_w ||
      (a.halo != 0 && a.halo != 2))
    return nullptr;
  return stencil_fn(a.tile_w, a.halo);
}

cudaError_t launch_stencil(const StencilArgs &sa, int grid, int block, size_t smem, cudaStream_t s) {
  cudaError_t e = stencil_prepare();
  if (e != cudaSuccess) return e;
  StencilArgs a = sa;
  const void *fn = stencil_launch_fn(a, block, smem);
  if (!fn) return cudaErrorInvalidValue;
  void *args[] = {(void *)&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t stencil_node(const StencilArgs &sa, int grid, int block, size_t smem, NodeChain &nc) {
  cudaError_t e = stencil_prepare();
  if (e != cudaSuccess) return e;
  StencilArgs a = sa;  // copied into the node's parameters by cudaGraphAddKernelNode
  const void *fn = stencil_launch_fn(a, block, smem);
  if (!fn) return cudaErrorInvalidValue;
  void *args[] = {(void *)&a};
  return nc.kernel(fn, dim3(grid), dim3(block), smem, args);
}

cudaError_t encode_u8_map(CUtensorMap *map, const void *base, int64_t W, int64_t H, int64_t D, int64_t pitch,
                          int box_w, int box_h) {
  EncodeTiledFn fn = get_encode();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)(pitch * H)};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------
// Allocation-free batched launch
//
// Some callers cannot allocate device memory (for example a host framework whose device memory is
// owned by its own pool allocator, or a loop that must not call cudaMalloc / cudaFree because those
// calls synchronise the device). For them the per-launch scratch of the stencil kernel — the tile
// counter, the status word, one tensor map and one instance record per instance, and the tile
// prefix sum — lives in the file-scope device array below, sized for kNoAllocMaxInstances
// instances (about 51 KB, held by every GPU that loads the library until the process exits).
// Every call reuses the same array: the counter and status word are cleared on each call, and two
// calls whose work overlaps on the GPU race on the array.
// ------------------------------------------------------------------------------------------
namespace {

struct NoAllocTables {
  CUtensorMap maps[kNoAllocMaxInstances];
  StencilInstance inst[kNoAllocMaxInstances];
  int64_t prefix[kNoAllocMaxInstances + 1];
  unsigned int queue;
  unsigned int status;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocTables)];

// Host staging copy of the tables (a static object: building them allocates nothing). The copies
// from it are made from pageable memory, so each call's copy has left it when the call returns.
static NoAllocTables g_noalloc_host;
static std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch for the current device, looked up once per device with
// that device current (host code cannot use the symbol itself as a device address).
cudaError_t noalloc_scratch_ptr(NoAllocTables **out) {
  static NoAllocTables *ptrs[256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (!ptrs[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    ptrs[dev] = reinterpret_cast<NoAllocTables *>(p);
  }
  *out = ptrs[dev];
  return cudaSuccess;
}

}  // namespace

size_t stencil_noalloc_scratch_bytes() { return sizeof(NoAllocTables); }

cudaError_t launch_stencil_noalloc(StencilArgs a, const uint8_t *in_base, uint8_t *out_base, const int64_t *desc,
                                   int64_t n, int sms, int cps, size_t smem, cudaStream_t s) {
  if (n < 1 || n > kNoAllocMaxInstances) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocTables *dev = nullptr;
  cudaError_t e = noalloc_scratch_ptr(&dev);
  if (e != cudaSuccess) return e;
  e = stencil_prepare();
  if (e != cudaSuccess) return e;
  NoAllocTables &h = g_noalloc_host;
  int64_t tiles = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t off = desc[5 * i], W = desc[5 * i + 1], H = desc[5 * i + 2], pitch = desc[5 * i + 3];
    e = encode_u8_map(&h.maps[i], in_base + off, W, H, 1, pitch, a.box_w, a.box_h);
    if (e != cudaSuccess) return e;
    StencilInstance &in = h.inst[i];
    in.in_off = off;
    in.out_off = off;
    in.W = (int32_t)W;
    in.H = (int32_t)H;
    in.D = 1;
    in.pitch_in = in.pitch_out = (int32_t)pitch;
    in.seed_xor = (uint32_t)desc[5 * i + 4];
    in.tiles_x = (int32_t)((W + a.tile_w - 1) / a.tile_w);
    in.tiles_y = (int32_t)((H + a.tile_h - 1) / a.tile_h);
    in.tile_base = tiles;
    h.prefix[i] = tiles;
    tiles += (int64_t)in.tiles_x * in.tiles_y;
  }
  h.prefix[n] = tiles;
  if (tiles >= (int64_t)UINT32_MAX - 1) return cudaErrorInvalidValue;
  e = cudaMemcpyAsync(dev->maps, h.maps, sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev->inst, h.inst, sizeof(StencilInstance) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev->prefix, h.prefix, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&dev->queue, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  a.maps = dev->maps;
  a.inst = dev->inst;
  a.tile_prefix = dev->prefix;
  a.in_base = in_base;
  a.out_base = out_base;
  a.queue = &dev->queue;
  a.status = &dev->status;
  a.total_tiles = tiles;
  a.ninst = (int32_t)n;
  const int64_t grid = tiles < (int64_t)sms * cps ? tiles : (int64_t)sms * cps;
  return launch_stencil(a, (int)(grid > 0 ? grid : 1), kBlock, smem, s);
}

cudaError_t stencil_noalloc_status(cudaStream_t s, unsigned int *out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocTables *dev = nullptr;
  cudaError_t e = noalloc_scratch_ptr(&dev);
  if (e != cudaSuccess) return e;
  unsigned int v = 0;
  e = cudaMemcpyAsync(&v, &dev->status, sizeof v, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *out = v;
  return e;
}

}  // namespace mrw
