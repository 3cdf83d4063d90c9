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
#include <mutex>

#include "mrw_internal.h"

namespace mrw {
namespace {

constexpr int kBlock = 256;
constexpr uint32_t kWaitPolls = 1u << 24;

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

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

__device__ __forceinline__ uint32_t apply_ops_px(const ChainOp *ops, int n, uint32_t p, int col, int W, uint32_t y,
                                                 const uint32_t *colhash, uint32_t seed_xor) {
  int kn = 0;
  for (int i = 0; i < n; ++i) {
    const ChainOp op = ops[i];
    if (op.kind == OP_SOLARISE) {
      p = p < 128u ? p : 255u - p;
    } else if (op.kind == OP_THRESH) {
      p = (p >= (op.t & 0xFFu) ? 1u : 0u) + (p >= ((op.t >> 8) & 0xFFu) ? 1u : 0u);
    } else if (op.kind == OP_NOISE) {
      uint32_t c;
      if (colhash != nullptr && kn < kMaxNoisePerGroup) {
        c = colhash[kn];
      } else {
        const uint32_t x = op.flip ? (uint32_t)(W - 1 - col) : (uint32_t)col;
        c = fmix32(fmix32(op.seed ^ seed_xor) ^ x);
      }
      const uint32_t hh = fmix32(c ^ y);
      const int q = (int)p + (int)(hh % 41u) - 20;
      p = (uint32_t)min(max(q, 0), 255);
      ++kn;
    }
  }
  return p;
}

__global__ void __launch_bounds__(kBlock) stencil_kernel(const __grid_constant__ StencilArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int BW = a.box_w, BH = a.box_h, TH = a.tile_h, TW = a.tile_w, h = a.halo;
  const int QP = (TW + 2 * h + 15) & ~15;  // Q row pitch
  const int nsq = TW + 2 * h;              // Q columns per tile (max)
  uint8_t *box[2] = {smem, smem + BH * BW};
  uint8_t *qt = smem + 2 * BH * BW;
  uint8_t *rt = qt + BH * QP;
  uint32_t *qcol = reinterpret_cast<uint32_t *>(rt + TH * TW);  // [kMaxNoisePerGroup][nsq]
  uint64_t *bar = reinterpret_cast<uint64_t *>(qcol + kMaxNoisePerGroup * ((nsq + 1) & ~1));
  __shared__ int64_t s_tile[2];
  __shared__ int s_fail;

  const int tid = threadIdx.x;
  const uint32_t box_bytes = (uint32_t)(BW * BH);
  uint32_t phase[2] = {0u, 0u};

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    const int64_t t = atomicAdd(a.queue, 1u);
    s_tile[0] = t;
    if (t < a.total_tiles) {
      const Tile g = locate(a, t);
      mbar_expect_tx(&bar[0], box_bytes);
      tma_load_3d(box[0], a.maps + g.inst, g.bx, g.by, g.z, &bar[0]);
    }
  }
  __syncthreads();

  int cur = 0;
  while (true) {
    const int64_t t = s_tile[cur];
    if (t >= a.total_tiles) break;
    const Tile g = locate(a, t);
    const StencilInstance inst = a.inst[g.inst];

    // Prefetch the next tile into the other buffer (free since the end of the previous iteration).
    if (tid == 0) {
      const int64_t tn = atomicAdd(a.queue, 1u);
      s_tile[cur ^ 1] = tn;
      if (tn < a.total_tiles) {
        const Tile gn = locate(a, tn);
        fence_proxy_async();
        mbar_expect_tx(&bar[cur ^ 1], box_bytes);
        tma_load_3d(box[cur ^ 1], a.maps + gn.inst, gn.bx, gn.by, gn.z, &bar[cur ^ 1]);
      }
      if (!mbar_wait_bounded(&bar[cur], phase[cur], a.wait_polls ? a.wait_polls - 1 : kWaitPolls)) s_fail = 1;
    }
    // Column hashes of the prefix's noise ops for this tile's Q columns.
    const int qcols = g.cols + 2 * h;
    {
      int kn = 0;
      for (int i = 0; i < a.npre && kn < kMaxNoisePerGroup; ++i) {
        if (a.pre[i].kind != OP_NOISE) continue;
        const uint32_t fs = fmix32(a.pre[i].seed ^ inst.seed_xor);
        for (int j = tid; j < qcols; j += kBlock) {
          const int gc = min(max(g.r0 - h + j, 0), g.W - 1);
          const uint32_t x = a.pre[i].flip ? (uint32_t)(g.W - 1 - gc) : (uint32_t)gc;
          qcol[kn * nsq + j] = fmix32(fs ^ x);
        }
        ++kn;
      }
    }
    __syncthreads();
    if (s_fail) break;
    phase[cur] ^= 1u;

    // Q tile: prefix applied to the clamped (replicated-edge) neighbourhood of the output tile.
    const uint8_t *bx = box[cur];
    const int qrows = g.rows + 2 * h;
    const uint32_t plane_row0 = (uint32_t)g.z * (uint32_t)g.H;
    for (int e = tid; e < qrows * qcols; e += kBlock) {
      const int i = e / qcols, j = e - i * qcols;
      const int gy = min(max(g.y0 - h + i, 0), g.H - 1);
      const int gc = min(max(g.r0 - h + j, 0), g.W - 1);
      const int ic = a.mpre ? g.W - 1 - gc : gc;
      uint32_t p = bx[(gy - g.by) * BW + (ic - g.bx)];
      uint32_t chv[kMaxNoisePerGroup];
#pragma unroll
      for (int k = 0; k < kMaxNoisePerGroup; ++k) chv[k] = qcol[k * nsq + j];
      p = apply_ops_px(a.pre, a.npre, p, gc, g.W, plane_row0 + (uint32_t)gy, chv, inst.seed_xor);
      qt[i * QP + j] = (uint8_t)p;
    }
    __syncthreads();

    const uint8_t *rsrc;  // R tile (blur output, or Q itself without a blur), pitch rpitch
    int rpitch;
    if (h == 2) {
      // 5x5 box sums: each thread owns 4 adjacent R columns and a run of rows; horizontal 5-sums
      // per Q row from two aligned words, vertical sums over a sliding window of five rows.
      const int quads = (g.cols + 3) >> 2;
      const int rows_per = 4;
      const int row_groups = (g.rows + rows_per - 1) / rows_per;
      for (int e = tid; e < quads * row_groups; e += kBlock) {
        const int jq = e % quads, rg = e / quads;
        const int i0 = rg * rows_per;
        const int ni = min(rows_per, g.rows - i0);
        uint32_t hs[rows_per + 4][4];
#pragma unroll
        for (int d = 0; d < rows_per + 4; ++d) {
          if (d < ni + 4) {
            const uint32_t *qw = reinterpret_cast<const uint32_t *>(qt + (i0 + d) * QP + 4 * jq);
            const uint32_t lo = qw[0], hi = qw[1];
            const uint32_t b0 = lo & 0xFF, b1 = (lo >> 8) & 0xFF, b2 = (lo >> 16) & 0xFF, b3 = lo >> 24;
            const uint32_t b4 = hi & 0xFF, b5 = (hi >> 8) & 0xFF, b6 = (hi >> 16) & 0xFF, b7 = hi >> 24;
            hs[d][0] = b0 + b1 + b2 + b3 + b4;
            hs[d][1] = hs[d][0] - b0 + b5;
            hs[d][2] = hs[d][1] - b1 + b6;
            hs[d][3] = hs[d][2] - b2 + b7;
          }
        }
#pragma unroll
        for (int i = 0; i < rows_per; ++i) {
          if (i < ni) {
            uint32_t outw = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const uint32_t s = hs[i][c] + hs[i + 1][c] + hs[i + 2][c] + hs[i + 3][c] + hs[i + 4][c];
              outw |= ((s + 12u) / 25u) << (8 * c);
            }
            *reinterpret_cast<uint32_t *>(rt + (i0 + i) * TW + 4 * jq) = outw;
          }
        }
      }
      __syncthreads();
      rsrc = rt;
      rpitch = TW;
    } else {
      rsrc = qt;
      rpitch = QP;
    }

    // Suffix and store: one 16-byte output segment per thread and row.
    const int segs = (g.cols + 15) >> 4;
    uint8_t *obase = a.out_base + inst.out_off + ((int64_t)g.z * g.H + g.y0) * inst.pitch_out + g.x0;
    for (int e = tid; e < segs * g.rows; e += kBlock) {
      const int i = e / segs, c = e - i * segs;
      const int nv = min(16, g.cols - 16 * c);
      uint8_t vb[16];
      const uint8_t *rrow = rsrc + i * rpitch;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        // output column x0+16c+k reads R local column (msuf: mirrored within the tile's span)
        const int lc = a.msuf ? g.cols - 1 - 16 * c - k : 16 * c + k;
        vb[k] = k < nv ? rrow[lc] : 0;
      }
      if (a.nsuf > 0) {
        const uint32_t y = plane_row0 + (uint32_t)(g.y0 + i);
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (k < nv) vb[k] = (uint8_t)apply_ops_px(a.suf, a.nsuf, vb[k], g.x0 + 16 * c + k, g.W, y, nullptr,
                                                    inst.seed_xor);
      }
      uint8_t *orow = obase + (int64_t)i * inst.pitch_out + 16 * c;
      if (nv == 16) {
        uint4 o;
        o.x = vb[0] | (vb[1] << 8) | (vb[2] << 16) | ((uint32_t)vb[3] << 24);
        o.y = vb[4] | (vb[5] << 8) | (vb[6] << 16) | ((uint32_t)vb[7] << 24);
        o.z = vb[8] | (vb[9] << 8) | (vb[10] << 16) | ((uint32_t)vb[11] << 24);
        o.w = vb[12] | (vb[13] << 8) | (vb[14] << 16) | ((uint32_t)vb[15] << 24);
        __stcs(reinterpret_cast<uint4 *>(orow), o);
      } else {
        for (int k = 0; k < nv; ++k) orow[k] = vb[k];
      }
    }
    __syncthreads();
    cur ^= 1;
  }

  if (s_fail && tid == 0) {
    atomicOr(a.status, 1u);
    // let the copies this CTA issued land before it leaves (bounded as well)
    if (s_tile[cur ^ 1] < a.total_tiles) (void)mbar_wait_bounded(&bar[cur ^ 1], phase[cur ^ 1]);
    (void)mbar_wait_bounded(&bar[cur], phase[cur]);
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

size_t stencil_smem_bytes(int tile_h, int tile_w, int halo) {
  const int BW = (tile_w + 2 * halo + 15 + 15) & ~15;
  const int BH = tile_h + 2 * halo;
  const int QP = (tile_w + 2 * halo + 15) & ~15;
  const int nsq = tile_w + 2 * halo;
  size_t b = (size_t)2 * BH * BW + (size_t)BH * QP + (size_t)tile_h * tile_w;
  b += (size_t)4 * kMaxNoisePerGroup * ((nsq + 1) & ~1);
  b = (b + 7) & ~(size_t)7;
  return b + 2 * sizeof(uint64_t);
}

cudaError_t stencil_prepare() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

cudaError_t launch_stencil(const StencilArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
  if (block != kBlock || smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = stencil_prepare();
  if (e != cudaSuccess) return e;
  stencil_kernel<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
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

}  // namespace mrw
