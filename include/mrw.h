/*
 * mrw.h — C ABI of the GB300 skeleton executor.
 *
 * A computation is a skeleton computational tree (SCT, Section 2 of Soldado,
 * Alexandre and Paulino, "Execution of Compound Multi-Kernel OpenCL
 * Computations in Multi-CPU/Multi-GPU Environments"): Pipeline, Map,
 * MapReduce and Loop nodes whose leaves are kernel stages (Table 1, "Marrow
 * constructs"). The tree is built bottom-up with the calls below, then
 * executed asynchronously on a CUDA stream; execution returns a future
 * (Section 2.1, "Execution request").
 *
 * Conventions for every entry point:
 *   - every call returns mrw_status; nothing aborts, throws or exits across
 *     the ABI; mrw_last_error() gives a thread-local message for the last
 *     failing call of this thread;
 *   - argument validation happens before anything is enqueued: a call that
 *     returns an error has launched nothing and allocated nothing it keeps;
 *   - device buffers belong to the caller; the executor borrows them until the
 *     future returned by the execute call has completed;
 *   - nodes are reference counted: creating a node gives the caller one
 *     reference; adding a node to a parent makes the parent hold its own
 *     reference; mrw_node_release drops the caller's;
 *   - streams are passed as `void*` holding a cudaStream_t (NULL = the legacy
 *     default stream); all work of one call is enqueued on that stream, on the
 *     CUDA device that is current when the call is made.
 *
 * The executor runs on ONE GPU: the paper's partitioning across devices
 * (Section 3.1) becomes partitioning across the SMs of that GPU.
 */
#ifndef MRW_H
#define MRW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRW_ABI_VERSION 1
#define MRW_MAX_DIMS 4
#define MRW_MAX_STAGES 64

/* ------------------------------------------------------------------------------------------ */
/* Status codes                                                                                */
/* ------------------------------------------------------------------------------------------ */
typedef enum mrw_status {
  MRW_OK = 0,
  MRW_ERR_INVALID_ARG = 1,  /* null pointer, unknown enum value, negative count            */
  MRW_ERR_SHAPE = 2,        /* buffer shapes disagree with each other or with the tree     */
  MRW_ERR_DTYPE = 3,        /* buffer element type is not the one the stage reads/writes   */
  MRW_ERR_CONSTRAINT = 4,   /* partitioning constraint violated (Section 3.1): epu not a
                               multiple of nu, pitch or pointer not 16-byte aligned, ...   */
  MRW_ERR_OOM = 5,          /* device or pinned-host allocation failed                     */
  MRW_ERR_CUDA = 6,         /* a CUDA runtime call failed; the message names it            */
  MRW_ERR_TIMEOUT = 7,      /* mrw_future_wait deadline passed; the future stays valid     */
  MRW_ERR_DEVICE = 8,       /* a kernel reported an error through its device status word
                               (a bounded wait gave up); the stream is still usable       */
  MRW_ERR_UNSUPPORTED = 9,  /* a tree shape or option the device path does not implement  */
  MRW_ERR_NOT_READY = 10    /* mrw_future_query: work still in flight                      */
} mrw_status;

/* ------------------------------------------------------------------------------------------ */
/* Data descriptors (Section 2.1 data types; Section 3.4 partitioning features)                */
/* ------------------------------------------------------------------------------------------ */
/* MRW_C64: complex single precision, interleaved (real, imaginary) float32 pairs, 8 bytes. */
typedef enum mrw_dtype { MRW_U8 = 0, MRW_I32 = 1, MRW_I64 = 2, MRW_F32 = 3, MRW_F64 = 4, MRW_BF16 = 5, MRW_C64 = 6 } mrw_dtype;

/* Where `data` lives. HOST buffers (pageable or pinned) are staged through device memory the
 * executor allocates per call and frees when the call's work is done, the way the paper's
 * Vector container hides data location and transfers (Section 2.1). Exception: when a whole image
 * tree fuses into one pointwise kernel and both image buffers are page-locked host memory mapped
 * into the device address space (e.g. cudaHostAlloc / torch pin_memory) with 16-byte aligned rows,
 * the kernel reads and writes them in place over the host link. */
typedef enum mrw_memory { MRW_MEM_DEVICE = 0, MRW_MEM_HOST = 1 } mrw_memory;

/* Transfer mode (Section 3.4): PARTITION splits the vector among the parallel executions by its
 * elementary partitioning unit; COPY gives every execution the whole vector (N-body positions). */
typedef enum mrw_transfer { MRW_PARTITION = 0, MRW_COPY = 1 } mrw_transfer;

typedef struct mrw_buffer {
  void *data;                   /* device or host address (see `memory`), borrowed           */
  mrw_dtype dtype;
  int32_t ndim;                 /* 1..4                                                      */
  int64_t shape[MRW_MAX_DIMS];  /* outermost first; an image is (H, W), a volume (D, H, W),
                                   an N-body state array (N, 4); every extent >= 1 (an empty
                                   buffer is refused with MRW_ERR_SHAPE before any launch)    */
  int64_t pitch;                /* bytes between consecutive rows (innermost dimension);
                                   0 = dense. Device image buffers need pitch % 16 == 0 and a
                                   16-byte-aligned `data`, and must span rows * pitch bytes  */
  int64_t epu;                  /* elementary partitioning unit in elements (Section 3.1);
                                   0 = default: one plane for images, one body for N-body    */
  mrw_transfer transfer;
  mrw_memory memory;
} mrw_buffer;

/* ------------------------------------------------------------------------------------------ */
/* Stages: the built-in kernel library (the leaves of an SCT)                                   */
/* ------------------------------------------------------------------------------------------ */
typedef enum mrw_stage_kind {
  /* u8 image stages; a buffer of shape (H, W) or (D, H, W) holds rows of W pixels and row y
   * of a volume is counted across planes. Section 4 benchmarks (Filter Pipeline, Segmentation). */
  MRW_ST_NOISE_HASH = 0,  /* p' = clamp(p + (hash32(seed, x, y) mod 41) - 20, 0, 255),
                             hash32(s,x,y) = F(F(F(s)^x)^y), F = MurmurHash3 fmix32; (x, y) are the
                             global column and row of the stage's input (Offset trait)          */
  MRW_ST_SOLARISE = 1,    /* p < 128 ? p : 255 - p                                              */
  MRW_ST_MIRROR_H = 2,    /* out[y][x] = in[y][W-1-x]                                           */
  MRW_ST_BOXBLUR5 = 3,    /* 5x5 box filter per plane, replicated edges, (sum + 12) / 25        */
  MRW_ST_THRESHOLD3 = 4,  /* label = (p >= t0) + (p >= t1); t0, t1 default 85, 170              */
  /* N-body stages on float32 (N, 4) arrays x = (pos, mass), v, a (Section 4, N-Body):          */
  MRW_ST_NBODY_ACCEL = 5, /* a_i = G sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2), d_ij = x_j - x_i  */
  MRW_ST_NBODY_KDK = 6,   /* one kick-drift-kick step: v += dt/2 a; x += dt v; a = a(x);
                             v += dt/2 a (a must hold a(x) on entry)                            */
  /* f32 Map stage (Section 4, Saxpy): y = alpha * x + y on two float32 vectors                 */
  MRW_ST_SAXPY = 7,
  /* Complex stages on rows of 65536 MRW_C64 values (Section 4, FFT pipelined with its inversion;
   * one row = one 512 KB elementary partitioning unit):                                         */
  MRW_ST_FFT = 8,         /* X[k] = sum_n x[n] exp(-2 pi i n k / N), not normalised              */
  MRW_ST_IFFT = 9         /* x[n] = (1/N) sum_k X[k] exp(+2 pi i n k / N)                        */
} mrw_stage_kind;

typedef struct mrw_stage_params {
  uint32_t seed;   /* NOISE_HASH                                                                  */
  int32_t t0, t1;  /* THRESHOLD3 thresholds; both 0 selects 85 and 170                            */
  float G;         /* NBODY_*: gravitational constant; 0 selects 1 / N                            */
  float eps;       /* NBODY_*: Plummer softening length                                           */
  float dt;        /* NBODY_KDK: time step                                                        */
  float alpha;     /* SAXPY                                                                       */
  int32_t nu;      /* elements of the partitioned vector each thread computes (Section 3.1 nu);
                      0 = the stage's default; must divide the buffer's epu                       */
  int32_t wg;      /* work-group (CTA) size the stage is bound to; 0 = executor's choice          */
} mrw_stage_params;

/* Merging functions of MapReduce (Section 3.4). The device path implements ADD: over a
 * THRESHOLD3-terminated map the result is the int64 count of each class (int64[3]); over any
 * other u8 map it is the int64 sum of the output values (int64[1]). */
typedef enum mrw_reduce_op { MRW_RED_ADD = 0, MRW_RED_SUB = 1, MRW_RED_MUL = 2, MRW_RED_DIV = 3 } mrw_reduce_op;

/* Loop state (Section 2.1: stop condition, carried data, global synchronisation). The device
 * evaluates the condition:
 *   MRW_LOOP_FOR: the body runs max_iters times; the iteration counter lives in device memory and
 *     an N-body loop is a CUDA graph whose conditional node re-reads it;
 *   MRW_LOOP_WHILE_CHANGED (image trees): the body runs again while its last run changed its input
 *     anywhere, at most max_iters times (a convergence loop, e.g. blurring to a fixed point). A
 *     device kernel compares each result with its input and sets the condition of a conditional
 *     WHILE node, so the number of iterations is decided on the GPU. At most one such loop per
 *     tree, not inside a MapReduce. */
typedef enum mrw_loop_kind { MRW_LOOP_FOR = 0, MRW_LOOP_WHILE_CHANGED = 1 } mrw_loop_kind;
typedef struct mrw_loop_state {
  int64_t max_iters;   /* 0 .. 1e8                                                              */
  int32_t kind;        /* mrw_loop_kind                                                         */
  int32_t global_sync; /* 1: every iteration sees all of the previous iteration's writes
                          (always the case on one GPU; kept for the paper's interface)          */
} mrw_loop_state;

/* ------------------------------------------------------------------------------------------ */
/* Execution configuration (the autotuner's search space; Algorithm 1 adapted to one GPU)       */
/* ------------------------------------------------------------------------------------------ */
typedef enum mrw_fusion { MRW_FUSE_ALL = 0, MRW_FUSE_NONE = 1 } mrw_fusion;

typedef struct mrw_config {
  int32_t fusion;      /* mrw_fusion: FUSE_ALL fuses every run of stages into one kernel; FUSE_NONE
                          runs one kernel per stage with materialised intermediates (the
                          kernel-per-stage baseline; a host-driven loop for Loop nodes)          */
  int32_t block;       /* threads per CTA (multiple of 32, 32..1024); 0 = default                */
  int32_t ctas_per_sm; /* resident CTAs per SM the grid is sized for; 0 = default                */
  int32_t tile_rows;   /* image: rows per CTA tile (stencil) ; N-body: bodies per thread (1,2,4) */
  int32_t tile_cols;   /* image: columns per CTA tile (stencil, multiple of 16, <= 256; a blur
                          tile is capped at 224 so its TMA box with halo fits 256 bytes)        */
  int32_t unroll;      /* image: 16-byte vectors each thread keeps in flight (1, 2, 4, 8)        */
  int32_t reserved[2]; /* must be 0                                                              */
} mrw_config;

/* ------------------------------------------------------------------------------------------ */
/* Opaque handles                                                                              */
/* ------------------------------------------------------------------------------------------ */
typedef struct mrw_node *mrw_node_t;
typedef struct mrw_future *mrw_future_t;
typedef struct mrw_model *mrw_model_t;

/* ------------------------------------------------------------------------------------------ */
/* Library                                                                                     */
/* ------------------------------------------------------------------------------------------ */
int32_t mrw_abi_version(void);
/* Thread-local message of this thread's last failing call ("" if none). Valid until the next
 * failing call on the same thread. */
const char *mrw_last_error(void);
const char *mrw_status_string(mrw_status s);

/* ------------------------------------------------------------------------------------------ */
/* SCT construction (Table 1: kernel, pipeline, loop, map, map_reduce)                          */
/* ------------------------------------------------------------------------------------------ */
/* A leaf: one kernel stage. `params` may be NULL (all defaults). */
mrw_status mrw_stage(mrw_stage_kind kind, const mrw_stage_params *params, mrw_node_t *out);
/* A leaf whose kernel the programmer writes (Section 2: the leaves of an SCT are user kernels): a u8
 * image stage given as CUDA C source that defines
 *     __device__ unsigned char <name>(unsigned char p, int x, int y, const unsigned int *u);
 * which maps the pixel p at column x and row y of the stage's input (global coordinates: rows of a
 * volume are counted across its planes, as for the noise stage; a mirror before the stage flips x)
 * to the stage's output pixel; u points at the 8 values of `params` (NULL: zeros). The function must
 * be pointwise and may call only device code it defines itself. `name` is a C identifier; `source`
 * and `name` are copied. The source is compiled here once as a check, with NVRTC (the CUDA
 * toolkit's run-time compiler, opened on first use); at execution, each group of consecutive
 * pointwise stages containing user stages (a blur ends a group) is compiled into one kernel that
 * applies all of them in registers, cached per generated source and device. User stages run in
 * mrw_execute on image trees (Map, Pipeline, Loop FOR, MapReduce over them); the batched calls and
 * WHILE_CHANGED loops return MRW_ERR_UNSUPPORTED for trees that contain one.
 * Errors: MRW_ERR_INVALID_ARG (NULL or empty argument, `name` not an identifier or longer than
 * 63 characters, `source` longer than 64 KiB); MRW_ERR_UNSUPPORTED (NVRTC not found, or the source
 * does not compile: mrw_last_error() holds the compiler's log). */
mrw_status mrw_stage_user(const char *name, const char *source, const uint32_t *params, mrw_node_t *out);
/* An empty Pipeline: a chain of control- and data-dependent subtrees (Section 2.1). */
mrw_status mrw_pipeline_create(mrw_node_t *out);
/* Append a new leaf stage to a pipeline. */
mrw_status mrw_pipeline_add_stage(mrw_node_t pipe, mrw_stage_kind kind, const mrw_stage_params *params);
/* Append an existing subtree (nesting, e.g. pipeline(K1, loop(K2), K3)); the pipeline retains it.
 * Adding a node to itself or to one of its descendants is rejected. */
mrw_status mrw_pipeline_add_node(mrw_node_t pipe, mrw_node_t child);
/* Map: apply `body` to independent partitions of the input (one partition per epu). */
mrw_status mrw_map(mrw_node_t body, mrw_node_t *out);
/* MapReduce: Map followed by a reduction with merging function `op` (see mrw_reduce_op). */
mrw_status mrw_mapreduce(mrw_node_t map_body, mrw_reduce_op op, mrw_node_t *out);
/* Loop: repeat `body` under `state` (Section 2.1, Loop). */
mrw_status mrw_loop(mrw_node_t body, const mrw_loop_state *state, mrw_node_t *out);
void mrw_node_retain(mrw_node_t n);
void mrw_node_release(mrw_node_t n);

/* ------------------------------------------------------------------------------------------ */
/* Execution (Table 1: run; returns a future)                                                   */
/* ------------------------------------------------------------------------------------------ */
/* Arguments by tree family:
 *   image trees (any nesting of Pipeline/Map/Loop over u8 stages): args[0] = input (u8),
 *     args[1] = output (u8, same shape, must not overlap the input); a MapReduce root may add
 *     args[2] = int64[3] class counts (THRESHOLD3 last) or int64[1] sum, overwritten; without
 *     args[2] (nargs = 2) the future holds the result (mrw_future_result; the plan, tuning and feature
 *     calls still take the three arguments);
 *   N-body trees (NBODY_ACCEL, NBODY_KDK, Pipeline/Loop of them): args = x, v, a, each float32
 *     (N, 4), updated in place;
 *   SAXPY: args = x, y (float32, same shape), y updated in place;
 *   FFT trees (FFT, IFFT, Pipeline/Map/Loop of them): args = x, y, each MRW_C64 of shape
 *     (nfft, 65536) or (65536), dense rows, 16-byte aligned device pointers; y = the stages applied
 *     to every row of x in order; y may
 *     be x itself (in place) but must not overlap it otherwise. FUSE_ALL runs up to 8 consecutive
 *     transforms in one launch (the values stay on chip or in L2 between transforms, so HBM sees
 *     each input read once and each output written once); FUSE_NONE runs one launch per
 *     transform. Up to as many rows as clusters of 8 CTAs run at once (36 on GB300), each row runs
 *     on such a cluster, two CTAs per SM; with more rows, a persistent grid splits every row into
 *     work items (16 columns or 16 lines of its 256 x 256 four-step matrix) whose values wait
 *     between phases in an L2-resident ring (a few tens of MB of device scratch per call; see
 *     mrw_fft_schedule_check; the first such call on a device also builds a 1 MB twiddle table
 *     that is kept until exit, so that call cannot be part of a stream capture). cfg->ctas_per_sm 1 asks for that form, 2 for the cluster form, 4
 *     for clusters of 8 with the exchange's values in tensor memory (three CTAs per SM), 3 for
 *     clusters of 16 CTAs (where the device allows that cluster size).
 * Every args[i] may be device or host memory (mrw_buffer.memory). The call is asynchronous:
 * it enqueues work on `stream` and returns a future in *out (release it with
 * mrw_future_release). `cfg` may be NULL (tuned or default configuration). A call that repeats
 * the calling thread's previous call (same tree, args, cfg, stream and device, and no tree,
 * knowledge-base or cost-model change in between) reuses that call's prepared launch when the plan
 * is a single pointwise kernel over device buffers, which skips the host's planning work. */
mrw_status mrw_execute(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfg,
                       void *stream, mrw_future_t *out);
/* As mrw_execute, and the future also records the call's device time for
 * mrw_future_elapsed_ms. Timing costs a pair of timing-enabled events on the stream around the
 * call (several microseconds per call on a busy stream), so mrw_execute records only an
 * ordering event. */
mrw_status mrw_execute_timed(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfg,
                             void *stream, mrw_future_t *out);

/* Batched execution (many independent instances of one image tree in one persistent launch):
 * instance i reads in_arena + desc[5i] and writes out_arena + desc[5i] with
 * desc[5i .. 5i+4] = {byte offset, W, H, pitch, noise seed}. Both arenas are device memory;
 * offsets must be multiples of 16, pitch a multiple of 16 and >= W, and every instance must lie
 * inside `arena_bytes`. Instance i's noise stages use (stage seed XOR desc seed of i), so a tree
 * built with seed 0 uses each instance's own seed. `desc` is a host array read before the call
 * returns; the launch (tensor maps, tile tables, graph) is cached per (tree, arenas, desc, cfg,
 * stream), so calls sharing a cache entry run in stream order. */
mrw_status mrw_execute_batched(mrw_node_t root, const uint8_t *in_arena, uint8_t *out_arena, int64_t arena_bytes,
                               const int64_t *desc, int64_t n, const mrw_config *cfg, void *stream,
                               mrw_future_t *out);

/* Allocation-free batched execution. The paper has no counterpart to this call; it serves callers
 * that must not allocate device memory — a host framework whose device memory belongs to its own
 * pool allocator, or a latency-critical loop in which cudaMalloc / cudaFree would synchronise the
 * device. It runs the same persistent stencil kernel as mrw_execute_batched, with the same
 * arguments and results, but allocates nothing: the kernel's scratch (tile counter, status word,
 * one tensor map and instance record per instance, tile prefix sum) lives in a file-scope device
 * array of about 51 KB sized for MRW_NOALLOC_MAX_INSTANCES instances, which every GPU that loads
 * the library holds until the process exits.
 *   - n must be 1..MRW_NOALLOC_MAX_INSTANCES; larger batches are rejected with
 *     MRW_ERR_INVALID_ARG ("takes 1 to 256 instances");
 *   - the tree must fuse into one kernel: image stages with at most one blur and at most 16
 *     pointwise stages on each side of it, cfg->fusion == MRW_FUSE_ALL (else MRW_ERR_UNSUPPORTED);
 *   - the call enqueues on `stream` and returns; it creates no future: synchronise the stream to
 *     wait. A tile wait that gives up its bound leaves that tile unwritten and sets the array's
 *     status word, which mrw_noalloc_status reads: check it after the work to know that every
 *     output byte was written;
 *   - every call reuses the one array, clearing its counter and status word on entry: calls whose
 *     work overlaps on the GPU (other streams, other host threads) race on it and must be
 *     serialised by the caller;
 *   - the call is not for CUDA graph capture: while `stream` is capturing it returns
 *     MRW_ERR_UNSUPPORTED and enqueues nothing (its table copies come from one shared host
 *     staging area that a replayed graph would read after later calls had changed it);
 *   - the first call on each device looks up the array's device address with that device current. */
#define MRW_NOALLOC_MAX_INSTANCES 256
mrw_status mrw_execute_batched_noalloc(mrw_node_t root, const uint8_t *in_arena, uint8_t *out_arena,
                                       int64_t arena_bytes, const int64_t *desc, int64_t n, const mrw_config *cfg,
                                       void *stream);
/* Status of the last mrw_execute_batched_noalloc call on the current device (no counterpart in the
 * paper): copies the array's status word out on `stream` behind the work already enqueued there,
 * waits for that stream and stores the word in *host_status (0: every tile wait ended in time).
 * Allocates nothing. Returns MRW_OK for 0, MRW_ERR_DEVICE when the last call gave up a wait (some
 * of its tiles are unwritten), MRW_ERR_INVALID_ARG for a NULL host_status, MRW_ERR_CUDA when the
 * copy fails. Query on the stream of the call, before the next call, which clears the word. */
mrw_status mrw_noalloc_status(void *stream, uint32_t *host_status);

/* Wait for a future: MRW_OK when the work finished, MRW_ERR_TIMEOUT if `timeout_ms` (< 0 =
 * forever) passed first (the future stays valid), MRW_ERR_DEVICE if a kernel gave up a bounded
 * wait, MRW_ERR_CUDA if the stream reported an error. */
mrw_status mrw_future_wait(mrw_future_t f, int64_t timeout_ms);
/* Non-blocking: MRW_OK when done, MRW_ERR_NOT_READY while running, errors as mrw_future_wait. */
mrw_status mrw_future_query(mrw_future_t f);
/* Device time between the first and the last enqueued operation of the call, in ms (after
 * completion). Only futures of mrw_execute_timed carry it; any other future gives
 * MRW_ERR_INVALID_ARG. */
mrw_status mrw_future_elapsed_ms(mrw_future_t f, float *ms);
/* The result of a MapReduce execution (Section 2.1: a run returns a future of the computation's
 * result; Table 1, run). Waits for the work (as mrw_future_wait with no deadline), then copies the
 * nresult int64 values to `host_dst` (host memory of at least `bytes` bytes; nresult = 3 class
 * counts for a THRESHOLD3-terminated map, else 1 value sum). Where the values come from:
 *   - the call had no args[2]: the future's own page-locked slot, filled by the call's work;
 *   - the call had args[2]: that buffer, read when this function runs (the future keeps no copy),
 *     so it must still hold the call's result.
 * Errors: MRW_ERR_INVALID_ARG (NULL argument, a tree without a reduction, bytes < 8 nresult),
 * and the errors of mrw_future_wait. May be called more than once, before mrw_future_release. */
mrw_status mrw_future_result(mrw_future_t f, void *host_dst, size_t bytes);
void mrw_future_release(mrw_future_t f);

/* The ticket schedule of the L2-ring FFT form (Section 4, FFT pipelined with its inversion, run as
 * a persistent grid; the paper has no such schedule): for nfft rows, nsteps transforms per launch
 * (1..8) and a grid of `ctas` CTAs, plans the slices and the ring, then checks on the host that every
 * work item (phase, row, 16-column or 16-line part) has exactly one ticket and that every item
 * waits only for items with smaller tickets, so that the persistent grid cannot deadlock. If `out`
 * is not NULL it receives 5 values: rows per slice, steps between a row's phases, ring rows (of
 * 512 KB each), grid CTAs and tickets. Launches nothing and needs no GPU. Errors:
 * MRW_ERR_UNSUPPORTED (no schedule: nfft < 1, nsteps outside 1..8, ctas < 1, or more than 2^31
 * tickets), MRW_ERR_CONSTRAINT (the check failed). */
mrw_status mrw_fft_schedule_check(int64_t nfft, int32_t nsteps, int32_t ctas, int64_t *out);

/* Describe the plan the executor would run for (root, args, cfg) as a JSON string: the fused
 * kernel groups, their stages, launch shapes and partitions. Writes at most `cap` bytes
 * (NUL-terminated); *needed receives the full length. Launches nothing. */
mrw_status mrw_plan_describe(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfg,
                             char *buf, int64_t cap, int64_t *needed);

/* ------------------------------------------------------------------------------------------ */
/* CPU + GPU co-execution with dynamic load balancing (Section 3.2 workload distribution         */
/* generator; Section 3.3, Dynamic Load Balancing and The Load Balancing Process)              */
/* ------------------------------------------------------------------------------------------ */
/* A balancer keeps, for one (tree, workload), the share of the rows the GPU runs, the load
 * balancing threshold lbt and the state of the adaptive binary search:
 *   - every co-executed run measures the GPU's and the host cores' times for their shares and
 *     their deviation dev = shortest / longest (1 = perfectly balanced);
 *   - isUnbalanced(dev) = 1 when dev / c_factor < max_dev, else 0, and
 *     lbt(n) = isUnbalanced(dev) * weight + lbt(n - 1) * (1 - weight), lbt(0) = 0;
 *   - profile construction (phase MRW_BAL_SEARCH): the whole work starts transferable; each run
 *     splits the transferable part evenly between the GPU and the host cores, then binds the half
 *     of the device that finished first to that device; the other half is the next transferable
 *     part (size / 2^n after n runs) until it is below `precision` (phase MRW_BAL_MONITOR);
 *   - when lbt reaches `trigger` (a persistent imbalance; three consecutive unbalanced runs from
 *     lbt = 0 at weight 2/3) the adaptive binary search moves work from the slower to the faster
 *     device: moves in one direction shift the search interval sideways by the transferable size
 *     (MRW_BAL_SHIFT), which doubles when more than two shifts in a row go the same way; the first
 *     move in the opposite direction returns to halving it (MRW_BAL_BISECT) until it is below
 *     `precision` again; then the balancer monitors (lbt reset to 0). */
typedef struct mrw_balancer *mrw_balancer_t;
typedef enum mrw_bal_phase { MRW_BAL_SEARCH = 0, MRW_BAL_MONITOR = 1, MRW_BAL_SHIFT = 2, MRW_BAL_BISECT = 3 } mrw_bal_phase;
typedef struct mrw_balance_params {
  double weight;      /* weight of the latest run in lbt; 0 = 2/3 (the paper's default)            */
  double max_dev;     /* balanced when (shortest / longest) / c_factor >= max_dev; 0 = 0.85         */
  double c_factor;    /* correction for computations that run best slightly unbalanced; 0 = 1      */
  double trigger;     /* lbt at which the load balancer starts moving work; 0 = 0.95               */
  double precision;   /* smallest transferable part of the searches (fraction of the work);
                         0 = 1/256                                                                 */
  double gpu_share;   /* initial share of the GPU in [0, 1] with a converged profile (phase
                         MONITOR); < 0 = profile construction from an even split                   */
  int32_t cpu_threads;/* host worker threads; 0 = every core the process may run on               */
  int32_t search_reps;/* runs at each share of the profile construction, the fastest time of each
                         side deciding (Algorithm 1's number of executions against fluctuations);
                         0 = 1                                                                     */
} mrw_balance_params;
typedef struct mrw_balance_report {
  double gpu_share;    /* share of the rows the GPU ran in this execution                         */
  int64_t gpu_rows, cpu_rows;
  double gpu_ms, cpu_ms;  /* device time of the GPU's share (CUDA events); wall time of the host
                             workers' share                                                        */
  double dev;          /* shortest / longest of the two times (1 if one side had no rows)          */
  int32_t unbalanced;  /* isUnbalanced(dev)                                                       */
  int32_t phase;       /* mrw_bal_phase after this execution                                      */
  double lbt;          /* after this execution                                                    */
  double next_share;   /* GPU share of the next execution                                         */
  double transferable; /* transferable part (fraction of the work) after this execution           */
} mrw_balance_report;
/* Errors: MRW_ERR_INVALID_ARG (NULL out, a parameter out of range: weight, max_dev, trigger,
 * precision in (0, 1], c_factor > 0, gpu_share <= 1, cpu_threads >= 0, search_reps 0 .. 64).
 * Starts the worker threads. */
mrw_status mrw_balancer_create(const mrw_balance_params *params, mrw_balancer_t *out);
void mrw_balancer_release(mrw_balancer_t b);
/* The balancer's bookkeeping for one run whose two shares took gpu_ms and cpu_ms (>= 0): updates
 * dev, lbt, the phase and the next share exactly as a co-executed run does, without running
 * anything (the search and the threshold on their own, e.g. for a caller that runs the shares
 * itself). *rep (may be NULL) receives the update; rep->gpu_share is the share that was run. */
mrw_status mrw_balancer_observe(mrw_balancer_t b, double gpu_ms, double cpu_ms, mrw_balance_report *rep);
/* The GPU share the next run will use. */
mrw_status mrw_balancer_share(mrw_balancer_t b, double *gpu_share);
/* Co-executes an image tree on host buffers: the GPU runs the first round(share x rows) rows (a
 * fused pointwise kernel reading and writing page-locked buffers in place, else staging its rows),
 * the host worker threads run the remaining rows at the same time (the same stage arithmetic; the
 * noise hash takes each row's global index, the Offset trait of Section 3.4), and a MapReduce's
 * partial results are merged on the host with + (Section 3.4 merging functions). Then the balancer
 * observes the two times (mrw_balancer_observe). Blocking: returns when both shares are done.
 * The tree must fuse into one pointwise kernel (noise, solarise, mirror, threshold3 stages under
 * Pipeline / Map / Loop, optionally a MapReduce root): args[0], args[1] host u8 images or volumes
 * (MRW_MEM_HOST); a MapReduce takes args[2] (int64[3] or int64[1], host or device) for the merged
 * result. Rows are the partitioning unit: the tree must be partitionable by rows (no blur).
 * Errors: as mrw_execute; MRW_ERR_UNSUPPORTED for device image buffers or a tree that does not
 * fuse into one pointwise kernel. */
mrw_status mrw_execute_coexec(mrw_balancer_t b, mrw_node_t root, const mrw_buffer *args, int32_t nargs,
                              const mrw_config *cfg, void *stream, mrw_balance_report *rep);

/* ------------------------------------------------------------------------------------------ */
/* Autotuner and knowledge base (Section 3.2: profile construction, Algorithm 1; knowledge base)*/
/* ------------------------------------------------------------------------------------------ */
typedef enum mrw_tune_mode {
  MRW_TUNE_EXHAUSTIVE = 0, /* time every valid candidate                                         */
  MRW_TUNE_PRUNED = 1,     /* Algorithm 1's ordered search: dimensions in order of likely benefit,
                              a dimension's remaining candidates are discarded as soon as one
                              fails to improve on the best so far                               */
  MRW_TUNE_MODEL = 2       /* ask the installed cost model (mrw_tune_set_model); no timing       */
} mrw_tune_mode;

/* Number of candidate configurations for (root, args) and, if `cfgs` is not NULL, up to `cap` of
 * them in a fixed order (index 0 is the default configuration). */
mrw_status mrw_tune_candidates(mrw_node_t root, const mrw_buffer *args, int32_t nargs, mrw_config *cfgs,
                               int32_t cap, int32_t *count);
/* Time `ncfg` configurations on the given (device) buffers: median of `reps` executions each,
 * after one warm-up, CUDA-event timed on `stream`; times_ms[i] < 0 marks an invalid config.
 * Blocks until done. The buffers' contents are overwritten as the tree's execution would. */
mrw_status mrw_tune_measure(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfgs,
                            int32_t ncfg, int32_t reps, void *stream, float *times_ms);
/* Pick a configuration for (root, args) by `mode`, record it in the knowledge base under the
 * tree's signature and the workload's shape, and return it. Later mrw_execute calls with
 * cfg == NULL use the recorded configuration. Blocks until done. */
mrw_status mrw_tune(mrw_node_t root, const mrw_buffer *args, int32_t nargs, mrw_tune_mode mode, int32_t reps,
                    void *stream, mrw_config *best, float *best_ms);
/* Knowledge base persistence: one text line per record {tree signature, workload signature,
 * config, best time, how it was obtained (exhaustive / pruned / model)}, Section 3.2 profiles. */
mrw_status mrw_kb_save(const char *path);
mrw_status mrw_kb_load(const char *path);
mrw_status mrw_kb_clear(void);
int64_t mrw_kb_size(void);

/* ------------------------------------------------------------------------------------------ */
/* Learned cost model (replaces the paper's interpolation-based configuration derivation,     */
/* Section 3.2): MLP 16 -> H -> H -> K, ReLU, bf16 weights, fp32 accumulation, fp32 master     */
/* weights and Adam state, all on the GPU.                                                      */
/* ------------------------------------------------------------------------------------------ */
#define MRW_NFEATURES 16
/* Features of a (tree, workload) pair: skeleton kind, stage counts by kind, bytes and ops per
 * element, log2 sizes, row width and alignment, dtype (host computation, no GPU needed). */
mrw_status mrw_features(mrw_node_t root, const mrw_buffer *args, int32_t nargs, float *feat16);
/* Create a model with K outputs and `hidden` units (<= 128), He-uniform weights from `seed`. */
mrw_status mrw_model_create(int32_t k, int32_t hidden, uint64_t seed, mrw_model_t *out);
void mrw_model_release(mrw_model_t m);
/* Number of float parameters (w1, b1, w2, b2, w3, b3 in that order, row-major [out][in]). */
int64_t mrw_model_num_params(mrw_model_t m);
/* Copy fp32 master parameters between host memory and the model (bf16 copies are refreshed,
 * Adam state is reset on set). Blocking. */
mrw_status mrw_model_set_params(mrw_model_t m, const float *host_params);
mrw_status mrw_model_get_params(mrw_model_t m, float *host_params);
/* Forward pass on device arrays: x float32 [n][16] -> y float32 [n][K] (predicted log times). */
mrw_status mrw_model_forward(mrw_model_t m, const float *x, int64_t n, float *y, void *stream);
/* Gradients of the mean squared loss over the n samples (device x [n][16], t [n][K]) into the
 * device array grads (num_params floats, same layout as the parameters); *loss (host) receives
 * the loss. Blocking. */
mrw_status mrw_model_gradients(mrw_model_t m, const float *x, const float *t, int64_t n, float *grads,
                               float *loss, void *stream);
/* One Adam step from device gradients (lr, b1 = 0.9, b2 = 0.999, eps = 1e-8). */
mrw_status mrw_model_adam_step(mrw_model_t m, const float *grads, float lr, void *stream);
/* Train for `epochs` passes over device data x [n][16], t [n][K] in shuffled minibatches of
 * `batch` samples (shuffle seeded by `seed`); *final_loss (host) = mean loss of the last epoch.
 * Blocking. */
mrw_status mrw_model_train(mrw_model_t m, const float *x, const float *t, int64_t n, int32_t epochs,
                           int32_t batch, float lr, uint64_t seed, void *stream, float *final_loss);
/* Install a model for MRW_TUNE_MODEL, with its K candidate configurations (copied). NULL removes it. */
mrw_status mrw_tune_set_model(mrw_model_t m, const mrw_config *cfgs, int32_t k);

#ifdef __cplusplus
}
#endif
#endif /* MRW_H */
