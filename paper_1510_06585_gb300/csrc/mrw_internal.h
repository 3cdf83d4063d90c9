// Internal interface between the host runtime (mrw_host.cpp) and the CUDA kernels.
// Not part of the public ABI (include/mrw.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "mrw.h"

namespace mrw {

// ------------------------------------------------------------------------------------------
// Image stages, as seen by the fused kernels
// ------------------------------------------------------------------------------------------
// OP_USER (a user-defined stage) never reaches the built-in kernels: groups that contain one run
// on a kernel compiled at run time (jit.cpp).
enum OpKind : int32_t { OP_NOISE = 0, OP_SOLARISE = 1, OP_MIRROR = 2, OP_BLUR = 3, OP_THRESH = 4, OP_USER = 5 };
enum RedKind : int32_t { RED_NONE = 0, RED_COUNT3 = 1, RED_SUM = 2 };

constexpr int kMaxChainOps = 16;     // pointwise ops fused into one kernel
constexpr int kMaxNoisePerGroup = 2; // noise ops whose column hashes stay in registers

// One pointwise op of a fused chain.
//   seed  : OP_NOISE seed (the kernels apply F = MurmurHash3 fmix32 to it, after XOR-ing in the
//           batched instance's seed in the stencil kernel)
//   flip  : the op's column coordinate is W-1-x (1) or x (0), x being the group's anchor column
//           (the output column for a chain; the blur's input column for a stencil prefix;
//           the output column for a stencil suffix)
//   t     : OP_THRESH thresholds, t0 | t1 << 8
struct ChainOp {
  int32_t kind;
  uint32_t seed;
  int32_t flip;
  uint32_t t;
};

// Fused pointwise chain over one u8 image or volume (rows of W pixels).
// Op sequences common enough that the kernels run them without walking the op list (mirror ops,
// which move no data, do not count). PAT_GENERIC: anything else, interpreted op by op.
enum OpPattern : int32_t {
  PAT_GENERIC = 0,
  PAT_NONE = 1,
  PAT_NOISE = 2,           // one noise op
  PAT_SOLARISE = 3,        // one solarise op
  PAT_NOISE_SOLARISE = 4,  // noise, then solarise
  PAT_THRESH = 5,          // one threshold op (its thresholds in the args' pattern_t)
};

// Pattern of ops[0, n) and, for PAT_THRESH, the op's thresholds in *t (host side).
inline int32_t op_pattern(const ChainOp *ops, int n, uint32_t *t) {
  int idx[2], m = 0;
  *t = 0;
  for (int i = 0; i < n; ++i) {
    if (ops[i].kind == OP_MIRROR) continue;
    if (m == 2) return PAT_GENERIC;
    idx[m++] = i;
  }
  if (m == 0) return PAT_NONE;
  const int k0 = ops[idx[0]].kind;
  if (m == 2) return k0 == OP_NOISE && ops[idx[1]].kind == OP_SOLARISE ? PAT_NOISE_SOLARISE : PAT_GENERIC;
  if (k0 == OP_NOISE) return PAT_NOISE;
  if (k0 == OP_SOLARISE) return PAT_SOLARISE;
  if (k0 == OP_THRESH) {
    *t = ops[idx[0]].t;
    return PAT_THRESH;
  }
  return PAT_GENERIC;
}

struct ChainArgs {
  const uint8_t *in;
  uint8_t *out;            // nullptr: reduce only
  int64_t in_pitch, out_pitch;
  int64_t rows;            // total rows (D * H)
  int64_t rows_parallel;   // row positions the threads cover at once (rows / unroll when blocked)
  int32_t W;
  int32_t col_vecs;        // ceil(W / 16)
  int32_t nops;
  int32_t mirror;          // parity of mirror ops in the chain: source column = W-1-x
  int32_t reduce;          // RedKind
  // row order of a thread: 0 = persistent (rows r0, r0 + rows_parallel, ...; one wave of CTAs),
  // 1 = blocked (unroll consecutive rows r0 * unroll + u; many short CTAs)
  int32_t blocked;
  unsigned long long *red; // RED_COUNT3: [3] counts; RED_SUM: [1]
  // MapReduce finish: with `partials` set (a per-stream workspace of kChainSlots sets of 3
  // accumulators, all zero between launches), CTA b adds into set b % kChainSlots and the finish
  // kernel launched next on the stream (launch_chain_finish) sums the sets into `red` and zeroes
  // them again; spreading the adds over the sets keeps thousands of CTAs from queueing on one
  // address. With `partials` null, CTAs add into a zeroed `red` (used when several launches
  // accumulate into one result).
  unsigned long long *partials;
  int64_t row0;            // global row of the first row (the Offset trait, for the noise hash)
  int32_t pattern;         // OpPattern of ops[0, nops) (set by launch_chain)
  uint32_t pattern_t;      // PAT_THRESH thresholds
  ChainOp ops[kMaxChainOps];
};

// A linear chain of CUDA graph nodes built through the graph API (each added node depends on the
// previous one). Plans that are replayed as graphs are built this way rather than by stream capture:
// while a stream of the process is capturing, another thread's device-wide synchronisation fails and
// invalidates the capture, so building by capture would break callers on other threads.
struct NodeChain {
  cudaGraph_t g = nullptr;
  cudaGraphNode_t last = nullptr;
  cudaError_t kernel(const void *func, dim3 grid, dim3 block, size_t smem, void **args) {
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void *>(func);
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned int)smem;
    kp.kernelParams = args;
    cudaGraphNode_t n = nullptr;
    const cudaError_t e = cudaGraphAddKernelNode(&n, g, last ? &last : nullptr, last ? 1 : 0, &kp);
    if (e == cudaSuccess) last = n;
    return e;
  }
  cudaError_t memset32(void *dst, unsigned int v, size_t count) {
    cudaMemsetParams mp = {};
    mp.dst = dst;
    mp.value = v;
    mp.elementSize = 4;
    mp.width = count;
    mp.height = 1;
    mp.pitch = 0;
    cudaGraphNode_t n = nullptr;
    const cudaError_t e = cudaGraphAddMemsetNode(&n, g, last ? &last : nullptr, last ? 1 : 0, &mp);
    if (e == cudaSuccess) last = n;
    return e;
  }
};

// Accumulator sets of the in-kernel MapReduce finish, and the largest grid of a chain launch.
constexpr int kChainSlots = 64;
constexpr int kMaxChainGrid = 1 << 22;

// Resident CTAs per SM of a chain-kernel variant (occupancy query, cached).
int chain_blocks_per_sm(int n_noise, bool mirror, int unroll, int block);
// n_noise: number of OP_NOISE entries (<= kMaxNoisePerGroup); unroll in {1, 2, 4, 8}.
cudaError_t launch_chain(const ChainArgs &a, int n_noise, int unroll, int grid, int block, cudaStream_t s);
// The same launch appended to a graph (no programmatic dependency there).
cudaError_t chain_node(const ChainArgs &a, int n_noise, int unroll, int grid, int block, NodeChain &nc);
// The MapReduce finish of a chain launch with a workspace: one CTA that sums the kChainSlots sets of
// `partials` into red[0, nout) and zeroes them; enqueue it right after that launch on the same stream.
cudaError_t launch_chain_finish(unsigned long long *partials, unsigned long long *red, int nout, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Stencil (5x5 box blur) groups and batched instances, TMA-staged tiles
// ------------------------------------------------------------------------------------------
struct StencilInstance {
  int64_t in_off, out_off;  // byte offsets from the arena bases
  int32_t W, H, D;          // plane width/height, planes
  int32_t pitch_in, pitch_out;
  uint32_t seed_xor;        // XOR-ed into every noise op's seed (batched instance seed)
  int64_t tile_base;        // first global tile index of this instance
  int32_t tiles_x, tiles_y;
};

struct StencilArgs {
  const CUtensorMap *maps;          // one 3-D map {W, H, D} per instance, device memory
  const StencilInstance *inst;      // device memory
  const int64_t *tile_prefix;       // [ninst + 1] device memory
  const uint8_t *in_base;
  uint8_t *out_base;
  unsigned int *queue;              // tile counter, zeroed before the launch
  unsigned int *status;             // status word (bounded waits); may be mapped host memory
  int64_t total_tiles;
  int32_t ninst;
  int32_t halo;                     // 2 with a blur, 0 for a pointwise-only group
  int32_t tile_h, tile_w;           // output tile (tile_w multiple of 16)
  int32_t box_w, box_h;             // TMA box
  int32_t npre, nsuf;               // prefix ops (before the blur) and suffix ops
  int32_t mpre, msuf;               // mirror parity of prefix and suffix
  int32_t reduce;                   // reserved (0)
  uint32_t wait_polls;              // 0: default bound; N > 0: give up a tile wait after N - 1 polls
                                    // (failure-detection tests set it through MRW_TEST_WAIT_POLLS)
  int32_t rows_kernel;              // 1: the row-streaming blur kernel (see stencil_rows_eligible):
                                    // tiles are strips of kRowsStrip columns by tile_h rows and the
                                    // maps' box is kRowsBoxW x kRowsChunk
  int32_t rows_cps;                 // row-streaming kernel: CTAs per SM the launch is sized for
                                    // (selects the variant budgeted for 4, or for 3, CTAs per SM)
  int32_t pre_pattern;              // row-streaming kernel: OpPattern of pre[0, npre) (set by
  uint32_t pre_pattern_t;           // launch_stencil) and its PAT_THRESH thresholds
  ChainOp pre[kMaxChainOps];
  ChainOp suf[kMaxChainOps];
};

// Row-streaming blur kernel: a warp streams strips of kRowsStrip output columns through a ring of
// kRowsBoxW x kRowsChunk TMA boxes. It runs groups with a blur, no suffix ops and at most
// kMaxNoisePerGroup noise stages in the prefix.
constexpr int kRowsStrip = 124;
constexpr int kRowsBoxW = 144;
constexpr int kRowsChunk = 8;
inline bool stencil_rows_eligible(int halo, int nsuf, int msuf, int n_noise_pre) {
  return halo == 2 && nsuf == 0 && msuf == 0 && n_noise_pre <= kMaxNoisePerGroup;
}
size_t stencil_rows_smem_bytes();
int stencil_rows_block();
// Resident CTAs per SM of the row-streaming kernel variant for a request of cps CTAs per SM
// (occupancy query, cached).
int stencil_rows_blocks_per_sm(int n_noise, int mirror, int cps);

// Tile widths the stencil kernel is compiled for (64, 128, 224): the one a request rounds to.
int stencil_tile_width(int requested);
// Shared-memory bytes the stencil kernel needs for a tile shape.
size_t stencil_smem_bytes(int tile_h, int tile_w, int halo);
cudaError_t launch_stencil(const StencilArgs &a, int grid, int block, size_t smem, cudaStream_t s);
// The same launch appended to a graph.
cudaError_t stencil_node(const StencilArgs &a, int grid, int block, size_t smem, NodeChain &nc);
// Set the kernels' shared-memory limits on the current device (once per device; also before a
// launch is added to a graph as a node).
cudaError_t stencil_prepare();
// Allocation-free batched launch: the tile counter, status word, tensor maps and instance tables
// live in a file-scope device array of k_stencil.cu (up to kNoAllocMaxInstances instances).
// `a` carries the ops and tile shape; the tables are built here from `desc` (n rows of
// {offset, W, H, pitch, seed}). Returns cudaErrorInvalidValue if n is out of range.
constexpr int kNoAllocMaxInstances = 256;
size_t stencil_noalloc_scratch_bytes();
cudaError_t launch_stencil_noalloc(StencilArgs a, const uint8_t *in_base, uint8_t *out_base, const int64_t *desc,
                                   int64_t n, int sms, int cps, size_t smem, cudaStream_t s);
// The status word of the allocation-free launch's array, read on stream `s` after the work enqueued
// before it (0: every tile wait of the last launch ended in time).
cudaError_t stencil_noalloc_status(cudaStream_t s, unsigned int *out);
// Encode a 3-D u8 tensor map for `base` with the stencil box of the given tile shape.
cudaError_t encode_u8_map(CUtensorMap *map, const void *base, int64_t W, int64_t H, int64_t D, int64_t pitch,
                          int box_w, int box_h);

// ------------------------------------------------------------------------------------------
// FFT stages: rows of kFftN complex float32 values, a cluster of kFftCluster CTAs per row
// ------------------------------------------------------------------------------------------
constexpr int kFftN = 65536;
constexpr int kFftCluster = 8;
constexpr int kFftMaxSteps = 8;
struct FftArgs {
  const float2 *in;              // nfft rows of kFftN values (16-byte aligned, dense)
  float2 *out;                   // same shape; may equal `in`
  int64_t nfft;
  int32_t nsteps;                // transforms applied in order, 1..kFftMaxSteps
  int32_t sign[kFftMaxSteps];    // +1 forward (kernel e^(-2 pi i nk/N)), -1 inverse (e^(+...), / N)
  unsigned int *status;          // 16-CTA kernel: set to 1 if a bounded wait gave up (may be null)
  uint32_t wait_polls;           // 16-CTA kernel: 0 = default bound; N > 0: give up after N - 1 polls
};
size_t fft_smem_bytes();
// Clusters that can be resident at once (0 if the launch configuration is not possible). tm: the
// form that keeps the exchange's values in TMEM instead of registers (three CTAs per SM).
int fft_max_clusters(bool tm);
cudaError_t launch_fft(const FftArgs &a, int clusters, bool tm, cudaStream_t s);
// Clusters of 16 CTAs (a non-portable cluster size), 16 of the 256 columns per CTA in 32 KB, and a
// second 32 KB buffer per CTA that the other CTAs fill with bulk copies between shared memories (the
// transposes of the four-step decomposition): three CTAs per SM. 0 clusters if the device cannot
// run them.
constexpr int kFft16Cluster = 16;
size_t fft16_smem_bytes();
int fft16_max_clusters();
cudaError_t launch_fft16(const FftArgs &a, int clusters, cudaStream_t s);

// The same chains with the four-step transposes exchanged through an L2-resident ring of rows in
// global memory: a persistent grid of CTAs of 16 kFftL2Block threads claims work items (phase p
// of row f, kFftL2Block of its columns or lines) from a ticket counter. See k_fft_l2.cu for the
// ticket order.
constexpr int kFftL2Block = 16;
constexpr int kFftL2Items = 256 / kFftL2Block;  // items per row and phase
struct FftSched {
  int64_t nfft;     // rows
  int64_t nslices;  // ceil(nfft / G)
  int32_t P;        // phases: transforms + 1
  int32_t G;        // rows per slice
  int32_t L;        // steps between a slice's consecutive phases (1 <= L <= nslices)
  int32_t pad;
};
struct FftL2Args {
  const float2 *in;        // nfft rows of kFftN values (16-byte aligned, dense)
  float2 *out;             // same shape; may equal `in`
  float2 *ring;            // ring_rows rows of kFftN values (256-byte aligned)
  unsigned int *done;      // nfft * P completion counters, zeroed by launch_fft_l2
  unsigned int *ticket;    // == done + nfft * P, zeroed with them
  unsigned int *status;    // set to 1 if a bounded wait gave up (may be null)
  const float2 *twiddle;   // fft_l2_twiddles: W_N^(k1 b) at [k1][b], then its inverse / N
  FftSched sc;
  int64_t ring_rows;
  int32_t nsteps;
  int32_t sign[kFftMaxSteps];
  uint32_t wait_polls;     // 0 = default bound; N > 0: give up a wait after N - 1 polls
};
struct FftL2Plan {
  FftSched sc;
  int64_t ring_rows;
  int ctas;                // grid size (at most the resident CTAs)
  size_t ring_bytes;       // ring_rows rows
  size_t counter_bytes;    // nfft * P + 1 counters
};
size_t fft_l2_smem_bytes();
// The per-device four-step twiddle table of the L2-ring kernel (built on first use, 1 MB, kept).
cudaError_t fft_l2_twiddles(const float2 **out);
int fft_l2_ctas_per_sm();  // resident CTAs per SM on the current device (0: cannot launch)
bool fft_l2_plan(int64_t nfft, int nsteps, int ctas, FftL2Plan *out);
bool fft_l2_schedule_ok(const FftSched &c, int64_t ring_rows);
int64_t fsch_total_tickets(const FftSched &c);  // work items of one launch (empty rows included)
cudaError_t launch_fft_l2(const FftL2Args &a, int ctas, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// N-body
// ------------------------------------------------------------------------------------------
struct LoopCtrl {
  unsigned long long iter;
  unsigned long long max_iters;
};

struct NBodyParams {
  float4 *x, *v, *a;
  int32_t n;
  float G, eps2, dt;
};

// a = G sum_j ... ; with kick: v += dt/2 a. bodies_per_thread in {1, 2, 4}.
cudaError_t launch_nbody_force(const NBodyParams &p, int kick, int bodies_per_thread, int grid, int block,
                               cudaStream_t s);
cudaError_t launch_nbody_drift(const NBodyParams &p, cudaStream_t s);
cudaError_t launch_nbody_kick(const NBodyParams &p, cudaStream_t s);
// Build and instantiate the device-controlled Loop graph: ctrl->iter = 0, then a conditional
// WHILE node whose body is {drift (advances the counter, sets the condition), force + kick}.
cudaError_t build_nbody_loop_graph(const NBodyParams &p, LoopCtrl *ctrl, int64_t iters, int bodies_per_thread,
                                   int grid, int block, cudaGraphExec_t *exec);

// ------------------------------------------------------------------------------------------
// SAXPY and helpers
// ------------------------------------------------------------------------------------------
// A Map of nstages saxpy stages fused into one pass: y := alpha[s] x + y for s in order (one fmaf per
// stage and element). x, y 16-byte aligned, n elements; unroll in {1, 2, 4, 8} float4 groups per
// thread (CTAs of 256 threads, one per 256 * unroll groups).
constexpr int kMaxSaxpyStages = 64;
struct SaxpyArgs {
  const float *x;
  float *y;
  int64_t n;
  int32_t nstages;
  float alpha[kMaxSaxpyStages];
};
cudaError_t launch_saxpy(const SaxpyArgs &a, int unroll, cudaStream_t s);
int saxpy_grid(int64_t n, int unroll);
// WHILE_CHANGED loops, as graph nodes: a := b where they differ and *changed := 1 if any byte
// differed; the control kernel counts the run and sets the WHILE node's condition
// (changed && iter < max); the init kernel zeroes the counter, words[0] (the changed flag) and
// words[1] (the body's status word).
cudaError_t compare_copy_node(const uint8_t *b, uint8_t *a, int64_t rows, int32_t W, int64_t pitch,
                              unsigned int *changed, int sms, NodeChain &nc);
cudaError_t while_control_node(LoopCtrl *ctrl, unsigned int *changed, cudaGraphConditionalHandle h, NodeChain &nc);
cudaError_t while_init_node(LoopCtrl *ctrl, unsigned int *words, unsigned long long max_iters, NodeChain &nc);

// ------------------------------------------------------------------------------------------
// Pointwise groups with user-defined stages, compiled at run time (jit.cpp)
// ------------------------------------------------------------------------------------------
// Parameter block of the generated kernel, passed by value; the generated source declares the
// same struct from the same field list (kUserArgsFields), so both sides agree on its layout.
constexpr int kUserParams = 8;  // 32-bit parameters of each op of the group
#define MRW_USER_ARGS_FIELDS                                                                        \
  const unsigned char *in;                                                                          \
  unsigned char *out;                                                                               \
  long long in_pitch, out_pitch, rows, row0;                                                        \
  int W;                                                                                            \
  unsigned int p[16][8];
struct UserChainArgs {
  MRW_USER_ARGS_FIELDS
};
#define MRW_STRINGIFY_(...) #__VA_ARGS__
#define MRW_STRINGIFY(...) MRW_STRINGIFY_(__VA_ARGS__)
constexpr const char *kUserArgsFields = MRW_STRINGIFY(MRW_USER_ARGS_FIELDS);
static_assert(kMaxChainOps == 16 && kUserParams == 8, "the field list spells out p[16][8]");

// Compiles `src` with NVRTC for sm_<arch>a without loading it; false with the compiler's message in
// *err if NVRTC is missing or the source does not compile.
bool jit_check(const std::string &src, int arch, std::string *err);
// The kernel `entry` of `src` compiled for sm_<arch>a and loaded on `device` (cached per source and
// device for the life of the process); false with a message in *err.
bool jit_kernel(const std::string &src, const char *entry, int device, int arch, cudaKernel_t *kernel,
                std::string *err);

// ------------------------------------------------------------------------------------------
// CPU + GPU co-execution (coexec.cpp)
// ------------------------------------------------------------------------------------------
// Sets this thread's mrw_last_error message and returns s.
mrw_status report_error(mrw_status s, const char *msg);
// One pointwise stage of the host workers' share (kind: OP_NOISE, OP_SOLARISE, OP_MIRROR, OP_THRESH).
struct HostChainOp {
  int32_t kind;
  uint32_t seed;
  uint32_t t;  // OP_THRESH thresholds, t0 | t1 << 8
};
// Rows [r0, r1) of an image through the stages, one row at a time (row r has global index y0 + r);
// red3 receives the rows' class counts (RED_COUNT3) or value sum in red3[0] (RED_SUM).
void host_chain_rows(const HostChainOp *ops, int nops, const uint8_t *in, int64_t in_pitch, uint8_t *out,
                     int64_t out_pitch, int W, int64_t y0, int64_t r0, int64_t r1, int reduce, uint64_t *red3);
// The balancer's host side: start the host share on its worker threads (returns at once), wait for
// it and merge its partial results; the share, lock and bookkeeping of a run.
mrw_status balancer_run_host_share(mrw_balancer *b, const HostChainOp *ops, int nops, const uint8_t *in,
                                   int64_t in_pitch, uint8_t *out, int64_t out_pitch, int W, int64_t y0,
                                   int64_t rows, int reduce);
void balancer_wait_host_share(mrw_balancer *b, uint64_t *red3);
double balancer_share_locked(mrw_balancer *b);
std::mutex &balancer_mutex(mrw_balancer *b);
void balancer_observe_locked(mrw_balancer *b, double gpu_ms, double cpu_ms, mrw_balance_report *rep);

// ------------------------------------------------------------------------------------------
// Cost-model MLP (bf16 weights, fp32 accumulation)
// ------------------------------------------------------------------------------------------
struct MlpDims {
  int32_t nin, hidden, k;
  int64_t off_w1, off_b1, off_w2, off_b2, off_w3, off_b3, nparams;
};
MlpDims mlp_dims(int nin, int hidden, int k);
cudaError_t launch_mlp_round_bf16(const float *master, uint16_t *bf, int64_t n, cudaStream_t s);
cudaError_t launch_mlp_forward(const MlpDims &d, const uint16_t *wbf, const float *x, int64_t n, float *y,
                               cudaStream_t s);
// grads must be zeroed by the caller; loss_acc (device float) accumulates sum of squared errors.
cudaError_t launch_mlp_backward(const MlpDims &d, const uint16_t *wbf, const float *x, const float *t,
                                const int32_t *idx, int64_t n, float scale, float *grads, float *loss_acc,
                                cudaStream_t s);
cudaError_t launch_mlp_adam(float *master, float *m, float *v, const float *g, int64_t n, float lr, float b1,
                            float b2, float eps, float bc1, float bc2, uint16_t *bf, cudaStream_t s);

}  // namespace mrw
