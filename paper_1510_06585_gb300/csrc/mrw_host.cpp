// Host runtime of the skeleton executor: the C ABI of include/mrw.h.
//
// Layers (Section 2 of the paper, re-cast for one GPU):
//   Library  — skeleton tree construction (Table 1): mrw_stage / pipeline / map / mapreduce / loop;
//   Scheduler— flattening the tree depth-first (Section 2, single-device execution model) into a
//              program, validating it against the buffers and the partitioning constraints
//              (Section 3.1), and grouping consecutive stages into fused kernels;
//   Task launcher — enqueueing the groups on the caller's stream, staging host buffers, and
//              returning a future backed by CUDA events (Section 2.1, run / Future);
//   Auto tuner + knowledge base — timing candidate configurations (Algorithm 1, adapted) and
//              recording the best per (tree, workload) (Section 3.2);
//   Cost model — a small MLP trained on the tuner's timings that derives a configuration for an
//              unseen pair (replacing the interpolation of Section 3.2, Configuration Derivation).
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cctype>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <random>
#include <sstream>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mrw.h"
#include "mrw_internal.h"

using namespace mrw;

// ============================================================================================
// Errors
// ============================================================================================
namespace {
thread_local std::string t_err;

mrw_status fail(mrw_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

mrw_status cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();  // clear a non-sticky error so the stream stays usable
  return fail(e == cudaErrorMemoryAllocation ? MRW_ERR_OOM : MRW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
  } while (0)

#define TRY(expr)                  \
  do {                             \
    mrw_status s_ = (expr);        \
    if (s_ != MRW_OK) return s_;   \
  } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

std::mutex g_mu;  // guards the caches below

struct DeviceInfo {
  int sms = 0;
  int arch = 0;  // compute capability major * 10 + minor
};
DeviceInfo device_info(int dev) {
  static std::map<int, DeviceInfo> cache;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  DeviceInfo d;
  cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  if (d.sms <= 0) d.sms = 1;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  d.arch = major * 10 + minor;
  cache[dev] = d;
  return d;
}

// ============================================================================================
// Status slots: a device word kernels can set, and a pinned host word it is copied into
// ============================================================================================
struct StatusSlot {
  unsigned int *dev = nullptr;
  unsigned int *host = nullptr;
  int idx = -1;
  int block = -1;
};

class StatusPool {
 public:
  mrw_status take(StatusSlot *out) {
    std::lock_guard<std::mutex> lk(mu_);
    if (free_.empty()) {
      // mapped pinned words: kernels write a failure straight into host memory, so a call needs
      // neither a reset nor a copy of its status word
      const int n = 1024;
      unsigned int *d = nullptr, *h = nullptr;
      if (cudaHostAlloc(&h, n * sizeof(unsigned int), cudaHostAllocMapped) != cudaSuccess)
        return fail(MRW_ERR_OOM, "pinned status words");
      memset(h, 0, n * sizeof(unsigned int));
      if (cudaHostGetDevicePointer((void **)&d, h, 0) != cudaSuccess) {
        cudaFreeHost(h);
        return fail(MRW_ERR_CUDA, "cudaHostGetDevicePointer(status words)");
      }
      const int b = (int)blocks_.size();
      blocks_.push_back({d, h});
      for (int i = n - 1; i >= 0; --i) free_.push_back({b, i});
    }
    auto [b, i] = free_.back();
    free_.pop_back();
    out->dev = blocks_[b].first + i;
    out->host = blocks_[b].second + i;
    out->idx = i;
    out->block = b;
    *out->host = 0;
    return MRW_OK;
  }
  void give(const StatusSlot &s) {
    if (s.idx < 0) return;
    *(volatile unsigned int *)s.host = 0u;
    std::lock_guard<std::mutex> lk(mu_);
    free_.push_back({s.block, s.idx});
  }

 private:
  std::mutex mu_;
  std::vector<std::pair<unsigned int *, unsigned int *>> blocks_;
  std::vector<std::pair<int, int>> free_;
};
StatusPool &status_pool() {
  static StatusPool p;
  return p;
}

// Page-locked slots of kResultSlot int64 values: the MapReduce result a future owns when its call
// was given no result buffer (args[2]). The call's staging copies the counts into the slot.
constexpr int kResultSlot = 4;
class ResultPool {
 public:
  mrw_status take(int64_t **out) {
    std::lock_guard<std::mutex> lk(mu_);
    if (free_.empty()) {
      const int n = 256;
      int64_t *h = nullptr;
      if (cudaHostAlloc(&h, n * kResultSlot * sizeof(int64_t), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(MRW_ERR_OOM, "pinned result slots");
      }
      memset(h, 0, n * kResultSlot * sizeof(int64_t));
      for (int i = n - 1; i >= 0; --i) free_.push_back(h + (int64_t)i * kResultSlot);
    }
    *out = free_.back();
    free_.pop_back();
    return MRW_OK;
  }
  void give(int64_t *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    free_.push_back(p);
  }

 private:
  std::mutex mu_;
  std::vector<int64_t *> free_;
};
ResultPool &result_pool() {
  static ResultPool p;
  return p;
}

// Accumulators of the chain kernel's MapReduce finish: one set per (device, stream), so launches
// that may overlap never share accumulators. The finish kernel leaves them at zero.
// A reducing chain launch and its finish kernel must be adjacent on their stream (the finish sums
// whatever the sets hold), so threads that share a stream enqueue the pair under this lock.
std::mutex g_reduce_mu;
struct ChainWs {
  unsigned long long *partials = nullptr;
};

mrw_status chain_workspace(int dev, cudaStream_t stream, ChainWs *out) {
  static std::map<std::pair<int, cudaStream_t>, ChainWs> cache;
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(dev, stream);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return MRW_OK;
  }
  if (cache.size() >= 256) return fail(MRW_ERR_UNSUPPORTED, "more than 256 streams used for MapReduce");
  ChainWs w;
  void *p = nullptr;
  const size_t bytes = sizeof(unsigned long long) * 3 * kChainSlots + 256;
  CU(cudaMalloc(&p, bytes));
  cudaError_t e = cudaMemset(p, 0, bytes);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_fail(e, "cudaMemset(workspace)");
  }
  w.partials = (unsigned long long *)p;
  cache[key] = w;
  *out = w;
  return MRW_OK;
}

// Timing-enabled event pairs for futures, reused instead of created per call.
class EventPool {
 public:
  mrw_status take(cudaEvent_t *a, cudaEvent_t *b) {
    std::lock_guard<std::mutex> lk(mu_);
    if (free_.size() >= 2) {
      *a = free_.back();
      free_.pop_back();
      *b = free_.back();
      free_.pop_back();
      return MRW_OK;
    }
    if (cudaEventCreate(a) != cudaSuccess) return cuda_fail(cudaErrorUnknown, "cudaEventCreate");
    if (cudaEventCreate(b) != cudaSuccess) {
      cudaEventDestroy(*a);
      return cuda_fail(cudaErrorUnknown, "cudaEventCreate");
    }
    return MRW_OK;
  }
  void give(cudaEvent_t a, cudaEvent_t b) {
    std::lock_guard<std::mutex> lk(mu_);
    if (free_.size() < 4096) {
      if (a) free_.push_back(a);
      if (b) free_.push_back(b);
    } else {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  }

 private:
  std::mutex mu_;
  std::vector<cudaEvent_t> free_;
};
EventPool &event_pool() {
  static EventPool p;
  return p;
}

// Ordering-only events (no timing) for overlapped staging, and two side streams per device.
std::vector<cudaEvent_t> *sync_event_pool() {
  static std::vector<cudaEvent_t> *pool = new std::vector<cudaEvent_t>();
  return pool;
}

mrw_status get_sync_event(cudaEvent_t *e) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!sync_event_pool()->empty()) {
      *e = sync_event_pool()->back();
      sync_event_pool()->pop_back();
      return MRW_OK;
    }
  }
  CU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return MRW_OK;
}

void put_sync_events(std::vector<cudaEvent_t> &v) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (cudaEvent_t e : v) sync_event_pool()->push_back(e);
  v.clear();
}

mrw_status side_streams(int dev, cudaStream_t *in, cudaStream_t *out) {
  static std::map<int, std::pair<cudaStream_t, cudaStream_t>> m;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = m.find(dev);
  if (it == m.end()) {
    cudaStream_t a, b;
    CU(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
    it = m.emplace(dev, std::make_pair(a, b)).first;
  }
  *in = it->second.first;
  *out = it->second.second;
  return MRW_OK;
}

// A non-blocking stream per device for copying a future's result out of device memory after its
// work has completed; callers hold g_result_mu from the copy to its synchronisation.
std::mutex g_result_mu;
mrw_status result_stream(int dev, cudaStream_t *out) {
  static std::map<int, cudaStream_t> m;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = m.find(dev);
  if (it == m.end()) {
    cudaStream_t s;
    CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    it = m.emplace(dev, s).first;
  }
  *out = it->second;
  return MRW_OK;
}

// A bounded cache of launch plans (CUDA graphs and the device memory they use). The key holds
// everything that decides what a plan enqueues, the stream included, so every launch of one entry
// is ordered on one stream; each use records the entry's `last_use` event behind its work. Evicting
// the least recently used entry waits for that event only (not for the device), outside the cache
// lock, and an entry a caller still holds is destroyed when that caller lets it go.
template <class Plan>
class PlanCache {
 public:
  using Ptr = std::shared_ptr<Plan>;
  explicit PlanCache(size_t cap) : cap_(cap) {}
  Ptr find(const std::string &key) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = m_.find(key);
    if (it == m_.end()) return nullptr;
    it->second.tick = ++tick_;
    return it->second.p;
  }
  // Adds `p` under `key` and returns the entry now cached there (another thread's, if it added the
  // same key first; `p` is then dropped).
  Ptr insert(const std::string &key, Ptr p) {
    Ptr evicted;
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto it = m_.find(key);
      if (it != m_.end()) {
        it->second.tick = ++tick_;
        evicted = std::move(p);
        return it->second.p;
      }
      if (m_.size() >= cap_) {
        auto lru = m_.begin();
        for (auto j = m_.begin(); j != m_.end(); ++j)
          if (j->second.tick < lru->second.tick) lru = j;
        evicted = std::move(lru->second.p);
        m_.erase(lru);
      }
      m_[key] = Entry{p, ++tick_};
    }
    return p;  // `evicted` is released here, after the lock
  }
  size_t size() {
    std::lock_guard<std::mutex> lk(mu_);
    return m_.size();
  }

 private:
  struct Entry {
    Ptr p;
    uint64_t tick = 0;
  };
  std::mutex mu_;
  std::map<std::string, Entry> m_;
  uint64_t tick_ = 0;
  size_t cap_;
};

// Wraps a built plan for a PlanCache: creates its last_use event; the deleter waits for that event
// and then frees the plan with `destroy`.
template <class Plan>
mrw_status make_cached(Plan &built, void (*destroy)(Plan &), std::shared_ptr<Plan> *out) {
  cudaEvent_t ev = nullptr;
  const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    destroy(built);
    return cuda_fail(e, "cudaEventCreate(plan)");
  }
  built.last_use = ev;
  *out = std::shared_ptr<Plan>(new Plan(built), [destroy](Plan *q) {
    cudaEventSynchronize(q->last_use);
    cudaEventDestroy(q->last_use);
    destroy(*q);
    delete q;
  });
  return MRW_OK;
}

// Records a plan's last_use event on the stream when the scope that enqueued work with it ends,
// whether or not every step succeeded.
struct RecordOnExit {
  cudaEvent_t ev;
  cudaStream_t stream;
  ~RecordOnExit() { cudaEventRecord(ev, stream); }
};

}  // namespace

// ============================================================================================
// Nodes (Section 2.1: SCT built bottom-up)
// ============================================================================================
enum NodeKind { N_STAGE = 0, N_PIPELINE = 1, N_MAP = 2, N_MAPREDUCE = 3, N_LOOP = 4 };

// A user-defined stage's device function (mrw_stage_user).
struct mrw_user_fn {
  std::string name, source;
};

struct mrw_node {
  std::atomic<int> refs{1};
  NodeKind kind = N_STAGE;
  mrw_stage_kind stage = MRW_ST_NOISE_HASH;
  mrw_stage_params params{};
  std::shared_ptr<const mrw_user_fn> user;  // set for a user-defined stage
  uint32_t uparams[kUserParams] = {};
  std::vector<mrw_node *> kids;
  mrw_reduce_op op = MRW_RED_ADD;
  mrw_loop_state loop{};
};

struct mrw_future {
  cudaEvent_t start = nullptr, done = nullptr;  // start is set (and done times) only when timed
  bool timed = false;
  int device = 0;
  StatusSlot slot;
  bool has_status = false;
  mrw_status deferred = MRW_OK;  // an error found while enqueueing after the first launch
  std::vector<cudaEvent_t> sync_events;  // cross-stream ordering events of an overlapped staging
  // MapReduce result (Section 2.1: the future of a run carries its result): nresult int64 values,
  // held in the future's own page-locked slot (the call had no args[2]) or in the caller's args[2]
  int32_t nresult = 0;
  int64_t *result_slot = nullptr;  // ResultPool slot, written by a copy enqueued with the call
  const void *result_src = nullptr;  // args[2] of the call, read when the result is asked for
  int result_mem = MRW_MEM_DEVICE;
};

namespace {

// Plan generation: advanced by every change that can alter what an execution of the same tree on
// the same arguments enqueues (a node created, grown or destroyed; the knowledge base or the
// installed cost model changed). A prepared launch is replayed only while it is unchanged.
std::atomic<uint64_t> g_plan_gen{1};
void bump_plan_gen() { g_plan_gen.fetch_add(1, std::memory_order_acq_rel); }

mrw_node *new_node(NodeKind k) {
  mrw_node *n = new (std::nothrow) mrw_node();
  if (n) n->kind = k;
  bump_plan_gen();
  return n;
}

void release_node(mrw_node *n) {
  if (!n) return;
  if (n->refs.fetch_sub(1) == 1) {
    for (mrw_node *c : n->kids) release_node(c);
    delete n;
    bump_plan_gen();
  }
}

bool contains(const mrw_node *root, const mrw_node *x) {
  if (root == x) return true;
  for (const mrw_node *c : root->kids)
    if (contains(c, x)) return true;
  return false;
}

bool valid_stage_kind(int k) { return k >= MRW_ST_NOISE_HASH && k <= MRW_ST_IFFT; }

mrw_stage_params default_params(mrw_stage_kind k, const mrw_stage_params *p) {
  mrw_stage_params q{};
  if (p) q = *p;
  if (k == MRW_ST_THRESHOLD3 && q.t0 == 0 && q.t1 == 0) {
    q.t0 = 85;
    q.t1 = 170;
  }
  return q;
}

// Structural signature of a tree (the paper's SCT unique identifier, Section 3.2 profiles).
void signature(const mrw_node *n, std::string &s) {
  char buf[160];
  switch (n->kind) {
    case N_STAGE: {
      const mrw_stage_params &p = n->params;
      if (n->user) {
        snprintf(buf, sizeof buf, "U%zx{", std::hash<std::string>()(n->user->name + '\n' + n->user->source));
        s += buf;
        for (int i = 0; i < kUserParams; ++i) {
          snprintf(buf, sizeof buf, "%s%u", i ? "," : "", n->uparams[i]);
          s += buf;
        }
        s += "}";
        return;
      }
      snprintf(buf, sizeof buf, "S%d{%u,%d,%d,%a,%a,%a,%a,%d,%d}", (int)n->stage, p.seed, p.t0, p.t1, p.G, p.eps,
               p.dt, p.alpha, p.nu, p.wg);
      s += buf;
      return;
    }
    case N_PIPELINE: s += "P("; break;
    case N_MAP: s += "M("; break;
    case N_MAPREDUCE: snprintf(buf, sizeof buf, "R%d(", (int)n->op); s += buf; break;
    case N_LOOP: snprintf(buf, sizeof buf, "L%lld,%d(", (long long)n->loop.max_iters, n->loop.kind); s += buf; break;
  }
  for (size_t i = 0; i < n->kids.size(); ++i) {
    if (i) s += ",";
    signature(n->kids[i], s);
  }
  s += ")";
}

// ============================================================================================
// Programs: the tree flattened depth-first (Section 2, single-device execution model)
// ============================================================================================
enum Family { F_NONE = 0, F_IMAGE = 1, F_NBODY = 2, F_SAXPY = 3, F_FFT = 4 };

struct ImgStage {
  int kind;  // OpKind
  uint32_t seed;
  uint32_t t;
  int nu, wg;
  std::shared_ptr<const mrw_user_fn> fn = nullptr;  // OP_USER: the device function
  std::array<uint32_t, kUserParams> up = {};        // OP_USER: its parameters
};

struct NbStep {
  int accel;  // 1: NBODY_ACCEL, 0: KDK steps
  int64_t iters;
  bool from_loop;
  float G, eps, dt;
  int nu, wg;
};

struct Program {
  Family fam = F_NONE;
  std::vector<ImgStage> img;
  int reduce = RED_NONE;
  bool stencil_in_row_map = false;  // a blur inside a Map whose partition is smaller than a plane
  bool has_map = false;
  std::vector<NbStep> nb;
  std::vector<float> alphas;
  std::vector<int> fft;  // transforms in order: +1 forward, -1 inverse
  int nu = 0, wg = 0;
  // a WHILE_CHANGED loop over img[while_begin, while_end), at most while_max runs (-1: none)
  int while_begin = -1, while_end = -1;
  int64_t while_max = 0;
};

mrw_status set_family(Program &p, Family f) {
  if (p.fam == F_NONE) p.fam = f;
  if (p.fam != f) return fail(MRW_ERR_UNSUPPORTED, "a tree mixes image, N-body, saxpy and FFT stages");
  return MRW_OK;
}

int op_kind_of(mrw_stage_kind k) {
  switch (k) {
    case MRW_ST_NOISE_HASH: return OP_NOISE;
    case MRW_ST_SOLARISE: return OP_SOLARISE;
    case MRW_ST_MIRROR_H: return OP_MIRROR;
    case MRW_ST_BOXBLUR5: return OP_BLUR;
    case MRW_ST_THRESHOLD3: return OP_THRESH;
    default: return -1;
  }
}

const mrw_node *last_leaf(const mrw_node *n) {
  while (n->kind != N_STAGE) {
    if (n->kids.empty()) return nullptr;
    n = n->kids.back();
  }
  return n;
}

mrw_status flatten(const mrw_node *n, Program &p, int depth, bool is_root, int64_t loop_mult) {
  if (depth > 64) return fail(MRW_ERR_UNSUPPORTED, "tree deeper than 64 levels");
  switch (n->kind) {
    case N_STAGE: {
      const mrw_stage_params &q = n->params;
      if (q.nu < 0 || q.wg < 0 || (q.wg && (q.wg % 32 || q.wg > 1024)))
        return fail(MRW_ERR_CONSTRAINT, "stage %d: wg must be a multiple of 32 up to 1024", (int)n->stage);
      if (n->user) {
        TRY(set_family(p, F_IMAGE));
        if ((int64_t)p.img.size() >= MRW_MAX_STAGES)
          return fail(MRW_ERR_UNSUPPORTED, "more than %d image stages after unrolling loops", MRW_MAX_STAGES);
        ImgStage st{OP_USER, 0, 0, q.nu, q.wg};
        st.fn = n->user;
        std::copy(n->uparams, n->uparams + kUserParams, st.up.begin());
        p.img.push_back(st);
        return MRW_OK;
      }
      const int ok = op_kind_of(n->stage);
      if (ok >= 0) {
        TRY(set_family(p, F_IMAGE));
        if ((int64_t)p.img.size() >= MRW_MAX_STAGES)
          return fail(MRW_ERR_UNSUPPORTED, "more than %d image stages after unrolling loops", MRW_MAX_STAGES);
        if (n->stage == MRW_ST_THRESHOLD3 && (q.t0 < 0 || q.t0 > 255 || q.t1 < 0 || q.t1 > 255 || q.t0 > q.t1))
          return fail(MRW_ERR_INVALID_ARG, "thresholds must satisfy 0 <= t0 <= t1 <= 255");
        p.img.push_back({ok, q.seed, (uint32_t)(q.t0 & 0xFF) | ((uint32_t)(q.t1 & 0xFF) << 8), q.nu, q.wg});
      } else if (n->stage == MRW_ST_NBODY_ACCEL || n->stage == MRW_ST_NBODY_KDK) {
        TRY(set_family(p, F_NBODY));
        if (!(q.eps > 0.f) || !std::isfinite(q.eps) || !std::isfinite(q.G) || !std::isfinite(q.dt) || q.G < 0.f)
          return fail(MRW_ERR_INVALID_ARG, "N-body stage needs finite G >= 0, dt and eps > 0");
        const bool accel = n->stage == MRW_ST_NBODY_ACCEL;
        if (!accel && !p.nb.empty() && !p.nb.back().accel && p.nb.back().G == q.G && p.nb.back().eps == q.eps &&
            p.nb.back().dt == q.dt && p.nb.back().from_loop == (loop_mult > 1)) {
          p.nb.back().iters += loop_mult;
        } else {
          p.nb.push_back({accel ? 1 : 0, accel ? 1 : loop_mult, loop_mult > 1 || !is_root, q.G, q.eps, q.dt, q.nu,
                          q.wg});
          if (accel && loop_mult > 1) return fail(MRW_ERR_UNSUPPORTED, "NBODY_ACCEL inside a Loop");
        }
      } else if (n->stage == MRW_ST_SAXPY) {
        TRY(set_family(p, F_SAXPY));
        for (int64_t i = 0; i < loop_mult; ++i) p.alphas.push_back(q.alpha);
      } else if (n->stage == MRW_ST_FFT || n->stage == MRW_ST_IFFT) {
        TRY(set_family(p, F_FFT));
        if ((int64_t)p.fft.size() + loop_mult > 4096) return fail(MRW_ERR_UNSUPPORTED, "more than 4096 transforms");
        for (int64_t i = 0; i < loop_mult; ++i) p.fft.push_back(n->stage == MRW_ST_FFT ? 1 : -1);
      } else {
        return fail(MRW_ERR_INVALID_ARG, "unknown stage kind %d", (int)n->stage);
      }
      if (q.nu) p.nu = q.nu;
      if (q.wg) p.wg = q.wg;
      return MRW_OK;
    }
    case N_PIPELINE:
      if (n->kids.empty()) return fail(MRW_ERR_INVALID_ARG, "empty pipeline");
      for (const mrw_node *c : n->kids) TRY(flatten(c, p, depth + 1, false, loop_mult));
      return MRW_OK;
    case N_MAP:
      p.has_map = true;
      return flatten(n->kids[0], p, depth + 1, false, loop_mult);
    case N_MAPREDUCE: {
      if (!is_root) return fail(MRW_ERR_UNSUPPORTED, "MapReduce must be the root of the executed tree");
      if (n->op != MRW_RED_ADD)
        return fail(MRW_ERR_UNSUPPORTED, "the device path implements the + merging function only");
      p.has_map = true;
      TRY(flatten(n->kids[0], p, depth + 1, false, loop_mult));
      if (p.fam != F_IMAGE) return fail(MRW_ERR_UNSUPPORTED, "MapReduce over a non-image map");
      const mrw_node *leaf = last_leaf(n->kids[0]);
      p.reduce = (leaf && leaf->stage == MRW_ST_THRESHOLD3) ? RED_COUNT3 : RED_SUM;
      return MRW_OK;
    }
    case N_LOOP: {
      const mrw_loop_state &st = n->loop;
      if (st.max_iters < 0 || st.max_iters > 100000000) return fail(MRW_ERR_INVALID_ARG, "loop max_iters out of range");
      if (st.kind != MRW_LOOP_FOR && st.kind != MRW_LOOP_WHILE_CHANGED)
        return fail(MRW_ERR_UNSUPPORTED, "loop kind %d", st.kind);
      if (st.kind == MRW_LOOP_WHILE_CHANGED) {
        if (p.while_begin >= 0) return fail(MRW_ERR_UNSUPPORTED, "more than one WHILE_CHANGED loop in a tree");
        if (loop_mult > 1) return fail(MRW_ERR_UNSUPPORTED, "a WHILE_CHANGED loop inside another loop");
        Program probe;
        TRY(flatten(n->kids[0], probe, depth + 1, false, 1));
        if (probe.fam != F_IMAGE || probe.while_begin >= 0)
          return fail(MRW_ERR_UNSUPPORTED, "WHILE_CHANGED loops run image trees");
        for (const ImgStage &st : probe.img)
          if (st.kind == OP_USER) return fail(MRW_ERR_UNSUPPORTED, "user-defined stages inside a WHILE_CHANGED loop");
        TRY(set_family(p, F_IMAGE));
        p.while_begin = (int)p.img.size();
        TRY(flatten(n->kids[0], p, depth + 1, false, 1));
        p.while_end = (int)p.img.size();
        p.while_max = st.max_iters;
        return MRW_OK;
      }
      if (st.max_iters == 0) return MRW_OK;
      if (loop_mult > 1 && st.max_iters > 1)
        return fail(MRW_ERR_UNSUPPORTED, "nested loops with more than one iteration each");
      Program probe;
      TRY(flatten(n->kids[0], probe, depth + 1, false, 1));
      if (probe.fam == F_IMAGE || probe.fam == F_SAXPY || probe.fam == F_FFT) {
        // pointwise / stencil bodies: iterations become consecutive stages (fused across iterations)
        for (int64_t i = 0; i < st.max_iters; ++i) TRY(flatten(n->kids[0], p, depth + 1, false, 1));
        return MRW_OK;
      }
      if (probe.fam == F_NBODY) {
        for (const NbStep &s : probe.nb)
          if (s.accel) return fail(MRW_ERR_UNSUPPORTED, "NBODY_ACCEL inside a Loop (the body must be KDK steps)");
        return flatten(n->kids[0], p, depth + 1, false, st.max_iters * loop_mult);
      }
      return MRW_OK;
    }
  }
  return fail(MRW_ERR_INVALID_ARG, "bad node");
}

// ============================================================================================
// Configurations: 16 candidates per family (the tuner's and the cost model's index space)
// ============================================================================================
struct Shape {
  int block, cps, unroll, tile_h, tile_w, bpt;
};
const Shape kShapes[8] = {
    {256, 8, 4, 32, 128, 2},   // default
    {256, 4, 2, 16, 128, 1},
    {128, 8, 8, 32, 64, 4},
    {512, 2, 4, 64, 64, 2},
    {256, 2, 1, 8, 256, 1},
    {128, 16, 2, 16, 64, 4},
    {128, 16, 8, 64, 128, 2},
    {256, 3, 4, 64, 128, 2},
};
const int kNbodyCps[8] = {1, 1, 1, 2, 2, 2, 4, 4};

mrw_config candidate(int i) {
  mrw_config c{};
  const Shape &s = kShapes[i % 8];
  c.fusion = i < 8 ? MRW_FUSE_ALL : MRW_FUSE_NONE;
  c.block = s.block;
  c.ctas_per_sm = s.cps;
  c.unroll = s.unroll;
  c.tile_rows = s.tile_h;
  c.tile_cols = s.tile_w;
  return c;
}

mrw_config nbody_candidate(int i) {
  mrw_config c{};
  const int s = i % 8;
  c.fusion = i < 8 ? MRW_FUSE_ALL : MRW_FUSE_NONE;
  c.block = 0;
  c.ctas_per_sm = kNbodyCps[s];
  c.tile_rows = (s % 3 == 0) ? 2 : (s % 3 == 1 ? 1 : 4);
  c.tile_cols = 0;
  c.unroll = 0;
  return c;
}

mrw_config default_config(Family f) { return f == F_NBODY ? nbody_candidate(0) : candidate(0); }

mrw_status check_config(const mrw_config &c) {
  if (c.fusion != MRW_FUSE_ALL && c.fusion != MRW_FUSE_NONE) return fail(MRW_ERR_INVALID_ARG, "bad fusion mode");
  if (c.block && (c.block % 32 || c.block < 32 || c.block > 1024)) return fail(MRW_ERR_INVALID_ARG, "bad block");
  if (c.ctas_per_sm < 0 || c.ctas_per_sm > 64) return fail(MRW_ERR_INVALID_ARG, "bad ctas_per_sm");
  if (c.unroll && c.unroll != 1 && c.unroll != 2 && c.unroll != 4 && c.unroll != 8)
    return fail(MRW_ERR_INVALID_ARG, "unroll must be 1, 2, 4 or 8");
  if (c.tile_rows < 0 || c.tile_rows > 252 || c.tile_cols < 0 || c.tile_cols > 256 || c.tile_cols % 16)
    return fail(MRW_ERR_INVALID_ARG, "bad tile shape");
  if (c.reserved[0] || c.reserved[1]) return fail(MRW_ERR_INVALID_ARG, "reserved config fields must be 0");
  return MRW_OK;
}

// ============================================================================================
// Buffers and argument validation
// ============================================================================================
int64_t elem_size(mrw_dtype t) {
  switch (t) {
    case MRW_U8: return 1;
    case MRW_BF16: return 2;
    case MRW_I32: case MRW_F32: return 4;
    case MRW_I64: case MRW_F64: case MRW_C64: return 8;
  }
  return 0;
}

struct View {       // a resolved 2-D view: rows of `width` elements, `pitch` bytes apart
  const mrw_buffer *b;
  int64_t width, rows, pitch, esize;
  int64_t numel() const { return width * rows; }
};

mrw_status view_of(const mrw_buffer &b, int idx, View *v) {
  if (!b.data) return fail(MRW_ERR_INVALID_ARG, "args[%d].data is NULL", idx);
  if (b.ndim < 1 || b.ndim > MRW_MAX_DIMS) return fail(MRW_ERR_SHAPE, "args[%d].ndim = %d", idx, b.ndim);
  const int64_t es = elem_size(b.dtype);
  if (!es) return fail(MRW_ERR_DTYPE, "args[%d]: unknown dtype", idx);
  if (b.memory != MRW_MEM_DEVICE && b.memory != MRW_MEM_HOST)
    return fail(MRW_ERR_INVALID_ARG, "args[%d]: bad memory kind", idx);
  int64_t rows = 1;
  for (int d = 0; d < b.ndim; ++d) {
    if (b.shape[d] < 1) return fail(MRW_ERR_SHAPE, "args[%d].shape[%d] = %lld", idx, d, (long long)b.shape[d]);
    if (d < b.ndim - 1) rows *= b.shape[d];
  }
  v->b = &b;
  v->width = b.shape[b.ndim - 1];
  v->rows = rows;
  v->esize = es;
  v->pitch = b.pitch ? b.pitch : v->width * es;
  if (v->pitch < v->width * es) return fail(MRW_ERR_SHAPE, "args[%d]: pitch smaller than a row", idx);
  return MRW_OK;
}

bool same_shape(const mrw_buffer &a, const mrw_buffer &b) {
  if (a.ndim != b.ndim) return false;
  for (int d = 0; d < a.ndim; ++d)
    if (a.shape[d] != b.shape[d]) return false;
  return true;
}

// ============================================================================================
// Staging: device copies of host buffers, released after the call's work (stream ordered)
// ============================================================================================
struct Staged {
  void *dev = nullptr;
  int64_t pitch = 0;
  bool copy_back = false;
  View src;
};

// A single fused chain launch prepared by an execute call: an image tree that plans into one
// pointwise kernel over device buffers. The next call of the same thread with the same tree,
// arguments, configuration, stream and device, and no change of the plan generation in between,
// replays it without planning again (the host cost of a small image is mostly planning and launch).
struct ChainReplay {
  bool valid = false;
  uint64_t gen = 0;
  const mrw_node *root = nullptr;
  int device = -1;
  cudaStream_t stream = nullptr;
  int32_t nargs = 0;
  mrw_buffer args[3];
  bool has_cfg = false;
  mrw_config cfg{};
  ChainArgs a{};
  int n_noise = 0, unroll = 1, grid = 0, block = 0;
  int finish_nout = 0;  // > 0: the MapReduce finish kernel follows the chain launch
};

struct Launch {  // everything one execute call enqueues
  cudaStream_t stream;
  int device;
  int sms;
  std::vector<void *> scratch;  // freed with cudaFreeAsync at the end
  std::vector<Staged> staged;
  std::vector<cudaEvent_t> *events = nullptr;  // ordering events to keep until the work is done
  ChainReplay *record = nullptr;  // set by execute: where a replayable chain launch is recorded
  bool recorded = false;

  mrw_status alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(scratch)");
    scratch.push_back(*p);
    return MRW_OK;
  }
  void free_all() {
    for (void *p : scratch) cudaFreeAsync(p, stream);
    scratch.clear();
  }
};

void configure_pool(int dev) {
  static std::map<int, bool> done;
  std::lock_guard<std::mutex> lk(g_mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool between calls
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

// Device view of args[i]: the buffer itself, or a staged device copy (rows padded to 16 bytes).
mrw_status resolve(Launch &L, const View &v, bool copy_in, bool copy_out, void **dev, int64_t *pitch) {
  if (v.b->memory == MRW_MEM_DEVICE) {
    *dev = v.b->data;
    *pitch = v.pitch;
    return MRW_OK;
  }
  Staged s;
  s.src = v;
  s.pitch = round_up(v.width * v.esize, 16);
  TRY(L.alloc(&s.dev, (size_t)(s.pitch * v.rows)));
  if (copy_in)
    CU(cudaMemcpy2DAsync(s.dev, s.pitch, v.b->data, v.pitch, v.width * v.esize, v.rows, cudaMemcpyHostToDevice,
                         L.stream));
  s.copy_back = copy_out;
  L.staged.push_back(s);
  *dev = s.dev;
  *pitch = s.pitch;
  return MRW_OK;
}

// Device address of a page-locked host buffer mapped into the device address space, if the buffer
// is one and its rows suit the streaming kernels (16-byte aligned start and pitch).
bool mapped_host(const View &v, void **dev) {
  if (v.b->memory != MRW_MEM_HOST || (uintptr_t)v.b->data % 16 || v.pitch % 16) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, v.b->data) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
  *dev = at.devicePointer;
  return true;
}

mrw_status copy_back(Launch &L) {
  for (const Staged &s : L.staged)
    if (s.copy_back)
      CU(cudaMemcpy2DAsync(s.src.b->data, s.src.pitch, s.dev, s.pitch, s.src.width * s.src.esize, s.src.rows,
                           cudaMemcpyDeviceToHost, L.stream));
  return MRW_OK;
}


// ============================================================================================
// Image plans: consecutive stages grouped into fused kernels
// ============================================================================================
struct Group {
  bool use_stencil = false;  // run by the stencil kernel (it has the blur, or the call is batched)
  bool user = false;         // has user-defined stages: a pointwise group compiled at run time
  bool blur = false;
  std::vector<ImgStage> pre, suf;  // pointwise stages before / after the blur
  int reduce = RED_NONE;           // fused MapReduce (chain groups only)
  bool reduce_only = false;        // a separate pass that reduces the previous group's output
};

int count_noise(const std::vector<ImgStage> &v) {
  int c = 0;
  for (const ImgStage &s : v) c += s.kind == OP_NOISE;
  return c;
}

int mirror_parity(const std::vector<ImgStage> &v) {
  int m = 0;
  for (const ImgStage &s : v) m ^= (s.kind == OP_MIRROR);
  return m;
}

// Fused: a group grows until a second blur, the op-count limit, or (chain groups) a third noise
// stage; the blur's position splits the group into prefix and suffix. Unfused: one stage per group
// (the kernel-per-stage execution), and a MapReduce reads the materialised labels in a pass of its own.
std::vector<Group> group_stages(const Program &p, bool fused, bool batched) {
  std::vector<Group> gs;
  if (!fused) {
    for (const ImgStage &s : p.img) {
      Group g;
      g.use_stencil = batched || s.kind == OP_BLUR;
      g.user = s.kind == OP_USER;
      g.blur = s.kind == OP_BLUR;
      if (!g.blur) g.pre.push_back(s);
      gs.push_back(g);
    }
  } else {
    Group cur;
    bool open = false;
    auto fresh = [&]() {
      cur = Group();
      cur.use_stencil = batched;
      open = true;
    };
    for (const ImgStage &s : p.img) {
      if (!open) fresh();
      if (s.kind == OP_BLUR) {
        if (cur.blur || cur.user) {  // user stages never run inside the blur kernels
          gs.push_back(cur);
          fresh();
        }
        cur.blur = true;
        cur.use_stencil = true;
        continue;
      }
      if (s.kind == OP_USER && cur.blur) {
        gs.push_back(cur);
        fresh();
      }
      std::vector<ImgStage> &list = cur.blur ? cur.suf : cur.pre;
      const bool full = (int)list.size() >= kMaxChainOps ||
                        (!cur.use_stencil && !cur.user && s.kind == OP_NOISE &&
                         count_noise(cur.pre) >= kMaxNoisePerGroup);
      if (full) {
        gs.push_back(cur);
        fresh();
      }
      (cur.blur ? cur.suf : cur.pre).push_back(s);
      cur.user = cur.user || s.kind == OP_USER;
    }
    if (open) gs.push_back(cur);
  }
  if (gs.empty()) {  // no stages: the output is a copy of the input
    Group g;
    g.use_stencil = batched;
    gs.push_back(g);
  }
  if (p.reduce != RED_NONE) {
    if (fused && !gs.back().use_stencil && !gs.back().user) {
      gs.back().reduce = p.reduce;
    } else {
      Group r;
      r.reduce_only = true;
      r.reduce = p.reduce;
      gs.push_back(r);
    }
  }
  return gs;
}

void fill_ops(const std::vector<ImgStage> &v, int anchor_parity, ChainOp *ops) {
  int before = 0;
  for (size_t i = 0; i < v.size(); ++i) {
    ops[i].kind = v[i].kind;
    ops[i].seed = v[i].seed;
    ops[i].t = v[i].t;
    ops[i].flip = anchor_parity ^ (before & 1);
    before += v[i].kind == OP_MIRROR;
  }
}

struct ImgGeom {
  int64_t W, H, D, rows;
};

struct ChainShape {
  int block, grid, unroll;
  int64_t rows_parallel;
  bool blocked;
  void apply(ChainArgs &a) const {
    a.rows_parallel = rows_parallel;
    a.blocked = blocked ? 1 : 0;
  }
};

// Launch shape of a chain group; each thread keeps one 16-byte column segment. Chains with noise
// stages run one wave of resident CTAs (the occupancy of the kernel variant caps ctas_per_sm) so a
// thread's per-column hash halves serve many rows. Chains without them are pure streaming: every
// thread takes `unroll` consecutive rows at a time in short CTAs that the hardware schedules as SMs
// free up (measured on GB300: a 128 MiB copy in this order runs about 5 % faster than the one-wave
// order). There the grid is capped at 8 x sms x ctas_per_sm CTAs; in a MapReduce group each CTA
// ends with a block reduction and three adds whose results it does not wait for.
ChainShape chain_shape(const mrw_config &cfg, int sms, int64_t W, int64_t rows, int wg, int n_noise,
                       bool mirror = false, bool query_occupancy = false) {
  ChainShape s;
  const int64_t col_vecs = (W + 15) / 16;
  if (n_noise == 0) {
    int block = wg ? wg : (cfg.block ? cfg.block : 256);
    int cps = cfg.ctas_per_sm ? cfg.ctas_per_sm : 8;
    if (block > 256) {  // compiled for at most 256 threads: keep threads per SM
      cps = std::max(1, cps * block / 256);
      block = 256;
    }
    s.block = block;
    s.unroll = cfg.unroll ? cfg.unroll : 4;
    s.blocked = true;
    const int64_t groups = (rows + s.unroll - 1) / s.unroll;
    const int64_t max_ctas = std::min<int64_t>((int64_t)8 * sms * cps, kMaxChainGrid);
    s.rows_parallel = std::max<int64_t>(1, std::min<int64_t>(groups, max_ctas * s.block / col_vecs));
    s.grid = (int)((s.rows_parallel * col_vecs + s.block - 1) / s.block);
    return s;
  }
  s.blocked = false;
  int block = wg ? wg : (cfg.block ? cfg.block : 256);
  int cps = cfg.ctas_per_sm ? cfg.ctas_per_sm : 64;
  if (block > 256) {  // the chain kernel is compiled for at most 256 threads: keep threads per SM
    cps = std::max(1, cps * block / 256);
    block = 256;
  }
  s.unroll = cfg.unroll ? cfg.unroll : 4;
  if (query_occupancy) cps = std::min(cps, chain_blocks_per_sm(n_noise, mirror, s.unroll, block));
  const int64_t target = std::min<int64_t>((int64_t)sms * cps * block, (int64_t)kMaxChainGrid * block);
  s.rows_parallel = std::max<int64_t>(1, std::min<int64_t>(rows, target / col_vecs));
  s.block = block;
  s.grid = (int)((s.rows_parallel * col_vecs + block - 1) / block);
  return s;
}

// Test hook of the failure-detection tests: make a bounded wait give up early.
uint32_t test_wait_polls() {
  const char *e = getenv("MRW_TEST_WAIT_POLLS");
  return e ? (uint32_t)strtoul(e, nullptr, 10) : 0u;
}

mrw_status run_chain(Launch &L, const Group &g, const uint8_t *in, int64_t ip, uint8_t *out, int64_t op,
                     const ImgGeom &geo, const mrw_config &cfg, int wg, unsigned long long *red) {
  ChainArgs a{};
  a.in = in;
  a.out = g.reduce_only ? nullptr : out;
  a.in_pitch = ip;
  a.out_pitch = op;
  a.rows = geo.rows;
  a.W = (int32_t)geo.W;
  a.col_vecs = (int32_t)((geo.W + 15) / 16);
  a.nops = (int32_t)g.pre.size();
  a.mirror = mirror_parity(g.pre);
  fill_ops(g.pre, a.mirror, a.ops);
  a.reduce = g.reduce;
  a.red = red;
  a.row0 = 0;
  if (g.reduce != RED_NONE) {  // finish the MapReduce in the kernel: no zeroing of `red` needed
    ChainWs ws;
    TRY(chain_workspace(L.device, L.stream, &ws));
    a.partials = ws.partials;
  }
  const ChainShape s = chain_shape(cfg, L.sms, geo.W, geo.rows, wg, count_noise(g.pre), a.mirror != 0, true);
  if (s.grid > kMaxChainGrid) return fail(MRW_ERR_UNSUPPORTED, "chain grid above %d CTAs", kMaxChainGrid);
  s.apply(a);
  const int nout = a.reduce == RED_COUNT3 ? 3 : 1;
  if (a.partials) {
    std::lock_guard<std::mutex> lk(g_reduce_mu);
    CU(launch_chain(a, count_noise(g.pre), s.unroll, s.grid, s.block, L.stream));
    CU(launch_chain_finish(a.partials, a.red, nout, L.stream));
  } else {
    CU(launch_chain(a, count_noise(g.pre), s.unroll, s.grid, s.block, L.stream));
  }
  if (L.record) {
    ChainReplay &r = *L.record;
    r.a = a;
    r.n_noise = count_noise(g.pre);
    r.unroll = s.unroll;
    r.grid = s.grid;
    r.block = s.block;
    r.finish_nout = a.partials ? nout : 0;
    L.recorded = true;
  }
  return MRW_OK;
}

struct StencilShape {
  int tile_h, tile_w, box_w, box_h, cps, block;
  size_t smem;
};

// A stencil group runs on the row-streaming kernel when it has a blur, no suffix and at most
// kMaxNoisePerGroup noise stages before the blur; otherwise on the 2-D tile kernel.
bool group_rows(const Group &g) {
  return stencil_rows_eligible(g.blur ? 2 : 0, (int)g.suf.size(), mirror_parity(g.suf), count_noise(g.pre));
}

void fill_stencil_ops(const Group &g, StencilArgs &a) {
  a.wait_polls = test_wait_polls();
  a.halo = g.blur ? 2 : 0;
  a.npre = (int32_t)g.pre.size();
  a.nsuf = (int32_t)g.suf.size();
  a.mpre = mirror_parity(g.pre);
  a.msuf = mirror_parity(g.suf);
  a.rows_kernel = group_rows(g) ? 1 : 0;
  fill_ops(g.pre, a.mpre, a.pre);
  fill_ops(g.suf, a.msuf, a.suf);
}

// Launch shape of a stencil group. The 2-D tile kernel takes tile_rows x tile_cols output tiles.
// The row-streaming kernel takes strips of kRowsStrip columns by 4 x tile_rows rows (a work item
// of one warp; the 4 halo rows it re-reads cost 4 / (4 x tile_rows) of the item).
StencilShape stencil_shape(const mrw_config &cfg, const StencilArgs &a) {
  StencilShape s;
  const int halo = a.halo;
  if (a.rows_kernel) {
    int nn = 0;
    for (int i = 0; i < a.npre; ++i) nn += a.pre[i].kind == OP_NOISE;
    s.tile_h = std::min(4096, std::max(8, 4 * (cfg.tile_rows ? cfg.tile_rows : 32)));
    s.tile_w = kRowsStrip;
    s.box_w = kRowsBoxW;
    s.box_h = kRowsChunk;
    const int want = cfg.ctas_per_sm ? cfg.ctas_per_sm : 8;
    s.cps = std::max(1, std::min(want, stencil_rows_blocks_per_sm(nn, a.mpre, want)));
    s.block = stencil_rows_block();
    s.smem = stencil_rows_smem_bytes();
    return s;
  }
  s.tile_h = cfg.tile_rows ? std::min(cfg.tile_rows, 252 - 2 * halo) : 32;
  s.tile_w = stencil_tile_width(cfg.tile_cols ? cfg.tile_cols : 128);
  s.tile_h = std::max(1, s.tile_h);
  s.box_w = (int)round_up(s.tile_w + 2 * halo + 15, 16);
  s.box_h = s.tile_h + 2 * halo;
  s.cps = std::min(8, cfg.ctas_per_sm ? cfg.ctas_per_sm : 4);
  s.block = 256;
  s.smem = stencil_smem_bytes(s.tile_h, s.tile_w, halo);
  return s;
}

void apply_shape(StencilArgs &a, const StencilShape &s) {
  a.rows_cps = s.cps;
  a.tile_h = s.tile_h;
  a.tile_w = s.tile_w;
  a.box_w = s.box_w;
  a.box_h = s.box_h;
}

// Persistent grid of a stencil launch over `tiles` work items: one item per CTA (tile kernel) or
// per warp (row-streaming kernel) at most, and at most cps CTAs per SM.
int stencil_grid(const StencilShape &s, const StencilArgs &a, int64_t tiles, int sms) {
  const int64_t per_cta = a.rows_kernel ? s.block / 32 : 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>((tiles + per_cta - 1) / per_cta, (int64_t)sms * s.cps));
}

// Device tables of a stencil launch: tensor maps, instances and the tile prefix sum.
struct StencilTables {
  std::vector<CUtensorMap> maps;
  std::vector<StencilInstance> inst;
  std::vector<int64_t> prefix;
  int64_t total = 0;
};

mrw_status upload_tables(Launch &L, const StencilTables &t, void **dev_maps, void **dev_inst, void **dev_prefix,
                         bool persistent, std::vector<void *> *owned) {
  const size_t mb = t.maps.size() * sizeof(CUtensorMap), ib = t.inst.size() * sizeof(StencilInstance),
               pb = t.prefix.size() * sizeof(int64_t);
  const size_t off_i = round_up((int64_t)mb, 256), off_p = off_i + round_up((int64_t)ib, 256);
  void *base = nullptr;
  if (persistent) {
    CU(cudaMalloc(&base, off_p + pb));
    owned->push_back(base);
  } else {
    TRY(L.alloc(&base, off_p + pb));
  }
  std::vector<uint8_t> host(off_p + pb);
  memcpy(host.data(), t.maps.data(), mb);
  memcpy(host.data() + off_i, t.inst.data(), ib);
  memcpy(host.data() + off_p, t.prefix.data(), pb);
  CU(cudaMemcpyAsync(base, host.data(), host.size(), cudaMemcpyHostToDevice, L.stream));
  if (persistent) CU(cudaStreamSynchronize(L.stream));  // `host` dies at return
  *dev_maps = base;
  *dev_inst = (uint8_t *)base + off_i;
  *dev_prefix = (uint8_t *)base + off_p;
  return MRW_OK;
}

mrw_status run_stencil_single(Launch &L, const Group &g, const uint8_t *in, int64_t ip, uint8_t *out, int64_t op,
                              const ImgGeom &geo, const mrw_config &cfg, unsigned int *status) {
  StencilArgs a{};
  fill_stencil_ops(g, a);
  const StencilShape s = stencil_shape(cfg, a);
  StencilTables t;
  t.maps.resize(1);
  CU(encode_u8_map(&t.maps[0], in, geo.W, geo.H, geo.D, ip, s.box_w, s.box_h));
  StencilInstance inst{};
  inst.in_off = 0;
  inst.out_off = 0;
  inst.W = (int32_t)geo.W;
  inst.H = (int32_t)geo.H;
  inst.D = (int32_t)geo.D;
  inst.pitch_in = (int32_t)ip;
  inst.pitch_out = (int32_t)op;
  inst.tiles_x = (int32_t)((geo.W + s.tile_w - 1) / s.tile_w);
  inst.tiles_y = (int32_t)((geo.H + s.tile_h - 1) / s.tile_h);
  inst.tile_base = 0;
  t.inst.push_back(inst);
  t.total = (int64_t)inst.tiles_x * inst.tiles_y * geo.D;
  t.prefix = {0, t.total};
  if (t.total >= (int64_t)1 << 31) return fail(MRW_ERR_UNSUPPORTED, "too many tiles");
  void *dm, *di, *dp;
  TRY(upload_tables(L, t, &dm, &di, &dp, false, nullptr));
  void *q;
  TRY(L.alloc(&q, 16));
  CU(cudaMemsetAsync(q, 0, 16, L.stream));
  a.maps = (const CUtensorMap *)dm;
  a.inst = (const StencilInstance *)di;
  a.tile_prefix = (const int64_t *)dp;
  a.in_base = in;
  a.out_base = out;
  a.queue = (unsigned int *)q;
  a.status = status;
  a.total_tiles = t.total;
  a.ninst = 1;
  apply_shape(a, s);
  CU(launch_stencil(a, stencil_grid(s, a, t.total, L.sms), s.block, s.smem, L.stream));
  return MRW_OK;
}

mrw_status validate_image_args(const Program &p, const mrw_buffer *args, int nargs, View *vin, View *vout,
                               View *vred) {
  const int need = p.reduce != RED_NONE ? 3 : 2;
  if (nargs != need) return fail(MRW_ERR_INVALID_ARG, "image tree takes %d arguments, got %d", need, nargs);
  TRY(view_of(args[0], 0, vin));
  TRY(view_of(args[1], 1, vout));
  if (args[0].dtype != MRW_U8 || args[1].dtype != MRW_U8) return fail(MRW_ERR_DTYPE, "image stages read/write u8");
  if (args[0].ndim < 2 || args[0].ndim > 3) return fail(MRW_ERR_SHAPE, "images are (H, W) or (D, H, W)");
  if (!same_shape(args[0], args[1])) return fail(MRW_ERR_SHAPE, "input and output shapes differ");
  if (vin->width > INT32_MAX / 2 || vin->rows > (int64_t)1 << 40) return fail(MRW_ERR_SHAPE, "image too large");
  for (int i = 0; i < 2; ++i) {
    const View &v = i ? *vout : *vin;
    if (v.b->memory == MRW_MEM_DEVICE && ((uintptr_t)v.b->data % 16 || v.pitch % 16))
      return fail(MRW_ERR_CONSTRAINT, "args[%d]: device images need a 16-byte aligned pointer and pitch", i);
  }
  // Partitioning constraints (Section 3.1): the elementary partitioning unit is a whole number of
  // rows, and the per-thread element count nu divides it.
  const int64_t plane = args[0].ndim == 3 ? args[0].shape[1] * vin->width : vin->rows * vin->width;
  const int64_t epu = args[0].epu ? args[0].epu : plane;
  if (epu % vin->width) return fail(MRW_ERR_CONSTRAINT, "epu %lld is not a whole number of rows", (long long)epu);
  if (p.nu && epu % p.nu) return fail(MRW_ERR_CONSTRAINT, "epu %lld is not a multiple of nu %d", (long long)epu, p.nu);
  bool blur = false;
  for (const ImgStage &s : p.img) blur |= s.kind == OP_BLUR;
  if (blur && p.has_map && epu % plane)
    return fail(MRW_ERR_CONSTRAINT, "a stencil inside a Map needs whole planes as partitions");
  // overlap: only a mirror-free, blur-free chain may run in place
  if (vin->b->memory == MRW_MEM_DEVICE && vout->b->memory == MRW_MEM_DEVICE) {
    const uintptr_t a0 = (uintptr_t)vin->b->data, a1 = a0 + vin->pitch * vin->rows;
    const uintptr_t b0 = (uintptr_t)vout->b->data, b1 = b0 + vout->pitch * vout->rows;
    const bool overlap = a0 < b1 && b0 < a1;
    bool mirror = false;
    for (const ImgStage &s : p.img) mirror |= s.kind == OP_MIRROR;
    if (overlap && (a0 != b0 || vin->pitch != vout->pitch || mirror || blur))
      return fail(MRW_ERR_INVALID_ARG, "output overlaps the input (only mirror- and blur-free chains run in place)");
  }
  if (p.reduce != RED_NONE) {
    TRY(view_of(args[2], 2, vred));
    const int64_t k = p.reduce == RED_COUNT3 ? 3 : 1;
    if (args[2].dtype != MRW_I64) return fail(MRW_ERR_DTYPE, "the MapReduce result is int64");
    if (vred->numel() != k) return fail(MRW_ERR_SHAPE, "the MapReduce result has %lld elements", (long long)k);
  }
  return MRW_OK;
}

ImgGeom geom_of(const mrw_buffer &b, const View &v) {
  ImgGeom g;
  g.W = v.width;
  g.rows = v.rows;
  if (b.ndim == 3) {
    g.D = b.shape[0];
    g.H = b.shape[1];
  } else {
    g.D = 1;
    g.H = v.rows;
  }
  return g;
}

// Run `gs` from src to dst: groups in order, intermediates in (at most two) stream-ordered
// scratch images; a reduce-only group reads the previous group's output.
// ---- groups with user-defined stages: one kernel generated per group and compiled at run time ----

// Source of the kernel for a pointwise group with user stages. A thread owns a 16-pixel segment of
// one row; each pixel goes through the group's stages in registers. The built-in stages are
// restated per pixel (noise: clamp(p + F(F(F(seed) ^ x) ^ y) mod 41 - 20) with F the MurmurHash3
// finaliser; solarise; threshold), the user functions each sit in a namespace of their own, and a
// mirror only flips the column coordinate of the stages after it (as in the chain kernel). All
// numeric parameters are kernel arguments, so the source depends only on the stage kinds, the
// mirrors and the user functions.
std::string user_chain_source(const Group &g) {
  const int parity = mirror_parity(g.pre);
  std::ostringstream o;
  o << "typedef unsigned int u32;\ntypedef unsigned char u8;\n"
    << "struct MrwUserArgs { " << kUserArgsFields << " };\n"
    << "__device__ __forceinline__ u32 mrw_fmix32(u32 h) {\n"
    << "  h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;\n  return h;\n}\n";
  int nu = 0;
  for (const ImgStage &st : g.pre)
    if (st.kind == OP_USER) o << "namespace mrw_user_" << nu++ << " {\n" << st.fn->source << "\n}\n";
  o << "__device__ __forceinline__ void mrw_unpack(u32 w, u8 *b) {\n"
    << "  b[0] = (u8)w; b[1] = (u8)(w >> 8); b[2] = (u8)(w >> 16); b[3] = (u8)(w >> 24);\n}\n"
    << "__device__ __forceinline__ u32 mrw_pack(const u8 *b) {\n"
    << "  return (u32)b[0] | (u32)b[1] << 8 | (u32)b[2] << 16 | (u32)b[3] << 24;\n}\n"
    << "extern \"C\" __global__ void __launch_bounds__(256) mrw_user_chain(const MrwUserArgs a) {\n"
    << "  const int W = a.W, segs = (W + 15) >> 4;\n"
    << "  const long long total = a.rows * segs, stride = (long long)gridDim.x * blockDim.x;\n"
    << "  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {\n"
    << "    const long long y = t / segs;\n"
    << "    const int x0 = (int)(t - y * segs) * 16, n = W - x0 < 16 ? W - x0 : 16;\n"
    << "    const u8 *src = a.in + y * a.in_pitch;\n"
    << "    u8 *dst = a.out + y * a.out_pitch;\n"
    << "    const u32 yg = (u32)(y + a.row0);\n"
    << "    u8 v[16];\n";
  if (!parity) {
    o << "    if (n == 16) {\n"
      << "      const uint4 q = *reinterpret_cast<const uint4 *>(src + x0);\n"
      << "      mrw_unpack(q.x, v); mrw_unpack(q.y, v + 4); mrw_unpack(q.z, v + 8); mrw_unpack(q.w, v + 12);\n"
      << "    } else {\n"
      << "#pragma unroll\n"
      << "      for (int k = 0; k < 16; ++k) v[k] = k < n ? src[x0 + k] : (u8)0;\n"
      << "    }\n";
  } else {
    o << "    if (n == 16 && (W & 15) == 0) {\n"
      << "      const uint4 q = *reinterpret_cast<const uint4 *>(src + (W - x0 - 16));\n"
      << "      u8 r[16];\n"
      << "      mrw_unpack(q.x, r); mrw_unpack(q.y, r + 4); mrw_unpack(q.z, r + 8); mrw_unpack(q.w, r + 12);\n"
      << "#pragma unroll\n"
      << "      for (int k = 0; k < 16; ++k) v[k] = r[15 - k];\n"
      << "    } else {\n"
      << "#pragma unroll\n"
      << "      for (int k = 0; k < 16; ++k) v[k] = k < n ? src[W - 1 - (x0 + k)] : (u8)0;\n"
      << "    }\n";
  }
  o << "#pragma unroll\n"
    << "    for (int k = 0; k < 16; ++k) {\n"
    << "      if (k >= n) continue;\n"
    << "      const int x = x0 + k;\n"
    << "      u32 p = v[k];\n";
  int before = 0, ui = 0;
  for (size_t i = 0; i < g.pre.size(); ++i) {
    const ImgStage &st = g.pre[i];
    const bool flip = (parity ^ (before & 1)) != 0;
    const char *col = flip ? "(W - 1 - x)" : "x";
    switch (st.kind) {
      case OP_MIRROR: ++before; break;
      case OP_NOISE:
        o << "      { const u32 h = mrw_fmix32(mrw_fmix32(mrw_fmix32(a.p[" << i << "][0]) ^ (u32)" << col
          << ") ^ yg); const int q = (int)p + (int)(h % 41u) - 20; p = q < 0 ? 0u : (q > 255 ? 255u : (u32)q); }\n";
        break;
      case OP_SOLARISE: o << "      p = p < 128u ? p : 255u - p;\n"; break;
      case OP_THRESH: o << "      p = (u32)(p >= a.p[" << i << "][0]) + (u32)(p >= a.p[" << i << "][1]);\n"; break;
      case OP_USER:
        o << "      p = (u32)mrw_user_" << ui++ << "::" << st.fn->name << "((u8)p, " << col << ", (int)yg, a.p[" << i
          << "]);\n";
        break;
      default: break;
    }
  }
  o << "      v[k] = (u8)p;\n"
    << "    }\n"
    << "    if (n == 16) {\n"
    << "      uint4 q;\n"
    << "      q.x = mrw_pack(v); q.y = mrw_pack(v + 4); q.z = mrw_pack(v + 8); q.w = mrw_pack(v + 12);\n"
    << "      *reinterpret_cast<uint4 *>(dst + x0) = q;\n"
    << "    } else {\n"
    << "#pragma unroll\n"
    << "      for (int k = 0; k < 16; ++k)\n"
    << "        if (k < n) dst[x0 + k] = v[k];\n"
    << "    }\n"
    << "  }\n"
    << "}\n";
  return o.str();
}

// The compiled kernel of a user group on the launch's device (compiled on first use, then cached).
mrw_status user_chain_kernel(const Launch &L, const Group &g, cudaKernel_t *k) {
  std::string err;
  if (!jit_kernel(user_chain_source(g), "mrw_user_chain", L.device, device_info(L.device).arch, k, &err))
    return fail(MRW_ERR_UNSUPPORTED, "%s", err.c_str());
  return MRW_OK;
}

// Compiles the kernels of every user group before anything is launched, so that a compile or load
// error leaves nothing enqueued.
mrw_status prepare_user_groups(const Launch &L, const std::vector<Group> &gs) {
  for (const Group &g : gs) {
    if (!g.user) continue;
    cudaKernel_t k;
    TRY(user_chain_kernel(L, g, &k));
  }
  return MRW_OK;
}

mrw_status run_user_chain(Launch &L, const Group &g, const uint8_t *in, int64_t ip, uint8_t *out, int64_t op,
                          const ImgGeom &geo, const mrw_config &cfg, int64_t row0) {
  cudaKernel_t k;
  TRY(user_chain_kernel(L, g, &k));
  UserChainArgs a{};
  a.in = in;
  a.out = out;
  a.in_pitch = ip;
  a.out_pitch = op;
  a.rows = geo.rows;
  a.row0 = row0;
  a.W = (int)geo.W;
  for (size_t i = 0; i < g.pre.size(); ++i) {
    const ImgStage &st = g.pre[i];
    if (st.kind == OP_NOISE) a.p[i][0] = st.seed;
    if (st.kind == OP_THRESH) {
      a.p[i][0] = st.t & 0xFF;
      a.p[i][1] = (st.t >> 8) & 0xFF;
    }
    if (st.kind == OP_USER)
      for (int j = 0; j < kUserParams; ++j) a.p[i][j] = st.up[j];
  }
  const int block = cfg.block > 0 ? cfg.block : 256;
  const int cps = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : 8;
  const int64_t work = geo.rows * ((geo.W + 15) / 16);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((work + block - 1) / block, (int64_t)L.sms * cps));
  void *args[] = {(void *)&a};
  CU(cudaLaunchKernel((const void *)k, dim3((unsigned)grid), dim3(block), args, 0, L.stream));
  return MRW_OK;
}

mrw_status run_groups(Launch &L, const std::vector<Group> &gs, const uint8_t *src, int64_t sp, uint8_t *dst,
                      int64_t dp_final, const ImgGeom &geo, const mrw_config &cfg, int wg, unsigned int *status,
                      bool *used_status, unsigned long long *red) {
  const int64_t tpitch = round_up(geo.W, 16);
  void *tmp[2] = {nullptr, nullptr};
  int n_out_groups = 0;
  for (const Group &g : gs) n_out_groups += !g.reduce_only;
  if (n_out_groups > 1) TRY(L.alloc(&tmp[0], (size_t)(tpitch * geo.rows)));
  if (n_out_groups > 2) TRY(L.alloc(&tmp[1], (size_t)(tpitch * geo.rows)));
  int k = 0;
  for (size_t gi = 0; gi < gs.size(); ++gi) {
    const Group &g = gs[gi];
    if (g.reduce_only) {
      TRY(run_chain(L, g, src, sp, nullptr, 0, geo, cfg, wg, red));
      continue;
    }
    ++k;
    const bool last = k == n_out_groups;
    uint8_t *d = last ? dst : (uint8_t *)tmp[(k - 1) & 1];
    const int64_t dp = last ? dp_final : tpitch;
    if (g.user) {
      TRY(run_user_chain(L, g, src, sp, d, dp, geo, cfg, 0));
    } else if (g.use_stencil) {
      TRY(run_stencil_single(L, g, src, sp, d, dp, geo, cfg, status));
      *used_status = true;
    } else {
      TRY(run_chain(L, g, src, sp, d, dp, geo, cfg, wg, g.reduce != RED_NONE ? red : nullptr));
    }
    src = d;
    sp = dp;
  }
  return MRW_OK;
}

// Host buffers, one fused pointwise group: stage the rows in chunks so that the copy-in of chunk
// c+1, the kernel on chunk c and the copy-out of chunk c-1 overlap (the paper's multi-buffered GPU
// execution platform, Section 2.2). Each chunk's kernel gets its global first row (Offset trait)
// and adds its counts into the zeroed result.
mrw_status enqueue_image_overlapped(Launch &L, const Group &g, const View &vin, const View &vout,
                                    const View *vred, const ImgGeom &geo, const mrw_config &cfg, int wg) {
  cudaStream_t s_in, s_out;
  TRY(side_streams(L.device, &s_in, &s_out));
  const int64_t pitch = round_up(geo.W, 16);
  void *din, *dout;
  TRY(L.alloc(&din, (size_t)(pitch * geo.rows)));
  TRY(L.alloc(&dout, (size_t)(pitch * geo.rows)));
  unsigned long long *red = nullptr;
  void *dred = nullptr;
  int64_t pred = 0;
  if (vred) {
    TRY(resolve(L, *vred, false, true, &dred, &pred));
    red = (unsigned long long *)dred;
    CU(cudaMemsetAsync(red, 0, (size_t)(vred->numel() * 8), L.stream));
  }
  const int64_t bytes = pitch * geo.rows;
  const int nch = (int)std::max<int64_t>(2, std::min<int64_t>(16, bytes / (4 << 20)));
  const int64_t crows = (geo.rows + nch - 1) / nch;
  cudaEvent_t ev_start;
  TRY(get_sync_event(&ev_start));
  L.events->push_back(ev_start);
  CU(cudaEventRecord(ev_start, L.stream));
  CU(cudaStreamWaitEvent(s_in, ev_start, 0));
  CU(cudaStreamWaitEvent(s_out, ev_start, 0));
  ChainArgs a{};
  a.W = (int32_t)geo.W;
  a.col_vecs = (int32_t)((geo.W + 15) / 16);
  a.nops = (int32_t)g.pre.size();
  a.mirror = mirror_parity(g.pre);
  fill_ops(g.pre, a.mirror, a.ops);
  a.reduce = g.reduce;
  a.red = red;
  a.in_pitch = a.out_pitch = pitch;
  for (int64_t r0 = 0; r0 < geo.rows; r0 += crows) {
    const int64_t nr = std::min(crows, geo.rows - r0);
    cudaEvent_t ev_in, ev_k;
    TRY(get_sync_event(&ev_in));
    L.events->push_back(ev_in);
    TRY(get_sync_event(&ev_k));
    L.events->push_back(ev_k);
    CU(cudaMemcpy2DAsync((uint8_t *)din + r0 * pitch, pitch, (const uint8_t *)vin.b->data + r0 * vin.pitch, vin.pitch,
                         geo.W, nr, cudaMemcpyHostToDevice, s_in));
    CU(cudaEventRecord(ev_in, s_in));
    CU(cudaStreamWaitEvent(L.stream, ev_in, 0));
    a.in = (const uint8_t *)din + r0 * pitch;
    a.out = (uint8_t *)dout + r0 * pitch;
    a.rows = nr;
    a.row0 = r0;
    const ChainShape s = chain_shape(cfg, L.sms, geo.W, nr, wg, count_noise(g.pre), a.mirror != 0, true);
    s.apply(a);
    CU(launch_chain(a, count_noise(g.pre), s.unroll, s.grid, s.block, L.stream));
    CU(cudaEventRecord(ev_k, L.stream));
    CU(cudaStreamWaitEvent(s_out, ev_k, 0));
    CU(cudaMemcpy2DAsync((uint8_t *)vout.b->data + r0 * vout.pitch, vout.pitch, (const uint8_t *)dout + r0 * pitch,
                         pitch, geo.W, nr, cudaMemcpyDeviceToHost, s_out));
  }
  cudaEvent_t ev_done;
  TRY(get_sync_event(&ev_done));
  L.events->push_back(ev_done);
  CU(cudaEventRecord(ev_done, s_out));
  CU(cudaStreamWaitEvent(L.stream, ev_done, 0));
  return MRW_OK;
}

// ============================================================================================
// WHILE_CHANGED loops: a cached CUDA graph {init; WHILE(cond) { body groups A -> B; a := b where
// they differ, flag; count, set cond }} whose condition is evaluated on the device
// ============================================================================================
Program sub_program(const Program &p, int b, int e) {
  Program q;
  q.fam = F_IMAGE;
  q.img.assign(p.img.begin() + b, p.img.begin() + e);
  q.nu = p.nu;
  q.wg = p.wg;
  q.has_map = p.has_map;
  return q;
}

struct Prepared {
  bool stencil = false;
  ChainArgs ca{};
  ChainShape cs{};
  int n_noise = 0;
  StencilArgs sa{};
  int grid = 0, block = 256;
  size_t smem = 0;
  unsigned int *queue = nullptr;
};

struct WhilePlan {
  void *mem = nullptr, *small = nullptr;
  uint8_t *A = nullptr, *B = nullptr;
  int64_t pitch = 0;
  LoopCtrl *ctrl = nullptr;
  unsigned int *words = nullptr;  // [0] changed, [1] status, [2 ..] tile queues
  std::vector<void *> owned;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t last_use = nullptr;  // recorded behind every use (PlanCache)
};

PlanCache<WhilePlan> &while_plans() {
  static PlanCache<WhilePlan> *c = new PlanCache<WhilePlan>(16);  // never destroyed: no CUDA calls at exit
  return *c;
}

void destroy_while_plan(WhilePlan &w) {
  if (w.exec) cudaGraphExecDestroy(w.exec);
  for (void *p : w.owned) cudaFree(p);
  if (w.mem) cudaFree(w.mem);
  if (w.small) cudaFree(w.small);
}

// Stencil launch with its tables in plan-owned memory (uploaded now, outside any capture).
mrw_status prepare_stencil(Launch &L, const Group &g, const uint8_t *in, int64_t ip, uint8_t *out, int64_t op,
                           const ImgGeom &geo, const mrw_config &cfg, unsigned int *status, unsigned int *queue,
                           std::vector<void *> *owned, Prepared *pr) {
  StencilArgs a{};
  fill_stencil_ops(g, a);
  const StencilShape s = stencil_shape(cfg, a);
  StencilTables t;
  t.maps.resize(1);
  CU(encode_u8_map(&t.maps[0], in, geo.W, geo.H, geo.D, ip, s.box_w, s.box_h));
  StencilInstance inst{};
  inst.W = (int32_t)geo.W;
  inst.H = (int32_t)geo.H;
  inst.D = (int32_t)geo.D;
  inst.pitch_in = (int32_t)ip;
  inst.pitch_out = (int32_t)op;
  inst.tiles_x = (int32_t)((geo.W + s.tile_w - 1) / s.tile_w);
  inst.tiles_y = (int32_t)((geo.H + s.tile_h - 1) / s.tile_h);
  t.inst.push_back(inst);
  t.total = (int64_t)inst.tiles_x * inst.tiles_y * geo.D;
  t.prefix = {0, t.total};
  void *dm, *di, *dp;
  TRY(upload_tables(L, t, &dm, &di, &dp, true, owned));
  a.maps = (const CUtensorMap *)dm;
  a.inst = (const StencilInstance *)di;
  a.tile_prefix = (const int64_t *)dp;
  a.in_base = in;
  a.out_base = out;
  a.queue = queue;
  a.status = status;
  a.total_tiles = t.total;
  a.ninst = 1;
  apply_shape(a, s);
  pr->stencil = true;
  pr->sa = a;
  pr->grid = stencil_grid(s, a, t.total, L.sms);
  pr->block = s.block;
  pr->smem = s.smem;
  pr->queue = queue;
  return MRW_OK;
}

void prepare_chain(const Group &g, const uint8_t *in, int64_t ip, uint8_t *out, int64_t op, const ImgGeom &geo,
                   const mrw_config &cfg, int sms, int wg, Prepared *pr) {
  ChainArgs &a = pr->ca;
  a = ChainArgs{};
  a.in = in;
  a.out = out;
  a.in_pitch = ip;
  a.out_pitch = op;
  a.rows = geo.rows;
  a.W = (int32_t)geo.W;
  a.col_vecs = (int32_t)((geo.W + 15) / 16);
  a.nops = (int32_t)g.pre.size();
  a.mirror = mirror_parity(g.pre);
  fill_ops(g.pre, a.mirror, a.ops);
  pr->n_noise = count_noise(g.pre);
  pr->cs = chain_shape(cfg, sms, geo.W, geo.rows, wg, pr->n_noise, a.mirror != 0, true);
  pr->cs.apply(a);
}

mrw_status build_while_plan(Launch &L, const Program &p, const ImgGeom &geo, const mrw_config &cfg, WhilePlan *wp) {
  const int64_t P = round_up(geo.W, 16), bytes = P * geo.rows;
  const Program body = sub_program(p, p.while_begin, p.while_end);
  const std::vector<Group> gs = group_stages(body, cfg.fusion == MRW_FUSE_ALL, false);
  if (gs.size() > 32) return fail(MRW_ERR_UNSUPPORTED, "loop body with more than 32 kernels");
  CU(cudaMalloc(&wp->mem, (size_t)(4 * bytes)));
  CU(cudaMalloc(&wp->small, 4096));
  CU(cudaMemset(wp->small, 0, 4096));
  wp->pitch = P;
  wp->A = (uint8_t *)wp->mem;
  wp->B = wp->A + bytes;
  uint8_t *T[2] = {wp->B + bytes, wp->B + 2 * bytes};
  wp->ctrl = (LoopCtrl *)wp->small;
  wp->words = (unsigned int *)((uint8_t *)wp->small + 256);
  std::vector<Prepared> prep(gs.size());
  const uint8_t *src = wp->A;
  for (size_t gi = 0; gi < gs.size(); ++gi) {
    const bool last = gi + 1 == gs.size();
    uint8_t *dst = last ? wp->B : T[gi & 1];
    if (gs[gi].use_stencil) {
      TRY(prepare_stencil(L, gs[gi], src, P, dst, P, geo, cfg, wp->words + 1, wp->words + 2 + gi, &wp->owned,
                          &prep[gi]));
    } else {
      prepare_chain(gs[gi], src, P, dst, P, geo, cfg, L.sms, p.wg, &prep[gi]);
    }
    src = dst;
  }
  CU(stencil_prepare());
  // the graph is built node by node (no stream capture)
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  // init: reset the counter, the changed flag and the status word
  NodeChain top;
  top.g = graph;
  if (e == cudaSuccess) e = while_init_node(wp->ctrl, wp->words, (unsigned long long)p.while_max, top);
  cudaGraphNode_t init_node = top.last;
  cudaGraphConditionalHandle handle{};
  cudaGraph_t bodyg = nullptr;
  if (e == cudaSuccess)
    e = cudaGraphConditionalHandleCreate(&handle, graph, p.while_max > 0 ? 1u : 0u, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond_node;
    e = cudaGraphAddNode(&cond_node, graph, &init_node, nullptr, 1, &cp);
    if (e == cudaSuccess) bodyg = cp.conditional.phGraph_out[0];
  }
  // body: the groups A -> B, then a := b where changed, then the control kernel
  if (e == cudaSuccess) {
    NodeChain body;
    body.g = bodyg;
    for (size_t gi = 0; e == cudaSuccess && gi < prep.size(); ++gi) {
      const Prepared &pr = prep[gi];
      if (pr.stencil) {
        e = body.memset32(pr.queue, 0u, 1);
        if (e == cudaSuccess) e = stencil_node(pr.sa, pr.grid, pr.block, pr.smem, body);
      } else {
        e = chain_node(pr.ca, pr.n_noise, pr.cs.unroll, pr.cs.grid, pr.cs.block, body);
      }
    }
    if (e == cudaSuccess) e = compare_copy_node(wp->B, wp->A, geo.rows, (int32_t)geo.W, P, wp->words, L.sms, body);
    if (e == cudaSuccess) e = while_control_node(wp->ctrl, wp->words, handle, body);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&wp->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "building the WHILE_CHANGED loop graph");
  return MRW_OK;
}

std::string image_program_key(const Program &p, const ImgGeom &geo, const mrw_config &c, int dev, cudaStream_t st) {
  std::ostringstream o;
  o << dev << "|" << (void *)st << "|" << geo.W << "x" << geo.H << "x" << geo.D << "|" << p.while_begin << ","
    << p.while_end << "," << p.while_max << "|" << c.fusion << "," << c.block << "," << c.ctas_per_sm << ","
    << c.tile_rows << "," << c.tile_cols << "," << c.unroll << "|";
  for (const ImgStage &s : p.img) o << s.kind << ":" << s.seed << ":" << s.t << ";";
  return o.str();
}

mrw_status enqueue_image_while(Launch &L, const Program &p, const View &vin, const View &vout, const ImgGeom &geo,
                               const mrw_config &cfg, unsigned int *status, bool *used_status) {
  const bool fused = cfg.fusion == MRW_FUSE_ALL;
  const Program pre = sub_program(p, 0, p.while_begin);
  const Program post = sub_program(p, p.while_end, (int)p.img.size());
  TRY(prepare_user_groups(L, group_stages(pre, fused, false)));  // user stages before / after the loop
  TRY(prepare_user_groups(L, group_stages(post, fused, false)));
  const std::string key = image_program_key(p, geo, cfg, L.device, L.stream);
  std::shared_ptr<WhilePlan> cached = while_plans().find(key);
  if (!cached) {
    WhilePlan built;
    mrw_status s = build_while_plan(L, p, geo, cfg, &built);
    if (s != MRW_OK) {
      destroy_while_plan(built);
      return s;
    }
    TRY(make_cached(built, destroy_while_plan, &cached));
    cached = while_plans().insert(key, cached);
  }
  const WhilePlan &wp = *cached;
  RecordOnExit used_until{wp.last_use, L.stream};
  void *din, *dout;
  int64_t pin, pout;
  TRY(resolve(L, vin, true, false, &din, &pin));
  TRY(resolve(L, vout, false, true, &dout, &pout));
  if (pre.img.empty()) {
    CU(cudaMemcpy2DAsync(wp.A, wp.pitch, din, pin, geo.W, geo.rows, cudaMemcpyDeviceToDevice, L.stream));
  } else {
    TRY(run_groups(L, group_stages(pre, fused, false), (const uint8_t *)din, pin, wp.A, wp.pitch, geo, cfg, p.wg,
                   status, used_status, nullptr));
  }
  CU(cudaGraphLaunch(wp.exec, L.stream));
  if (status) {
    CU(cudaMemcpyAsync(status, wp.words + 1, sizeof(unsigned int), cudaMemcpyDefault, L.stream));
    *used_status = true;
  }
  if (post.img.empty()) {
    CU(cudaMemcpy2DAsync(dout, pout, wp.A, wp.pitch, geo.W, geo.rows, cudaMemcpyDeviceToDevice, L.stream));
  } else {
    TRY(run_groups(L, group_stages(post, fused, false), wp.A, wp.pitch, (uint8_t *)dout, pout, geo, cfg, p.wg,
                   status, used_status, nullptr));
  }
  return MRW_OK;
}

// One chain group over two host image buffers: such a plan reads and writes page-locked buffers in
// place, or stages the rows in overlapped chunks (chunked_staging).
bool host_one_chain(const std::vector<Group> &gs, const View &vin, const View &vout) {
  return gs.size() == 1 && !gs[0].use_stencil && !gs[0].user && vin.b->memory == MRW_MEM_HOST &&
         vout.b->memory == MRW_MEM_HOST;
}

// Whether an execution stages its host rows in overlapped chunks (enqueue_image_overlapped): one
// chain group over host buffers that are not both mapped page-locked memory, at least 64 rows and
// 8 MiB. Such a plan reduces by adds into the zeroed result, with no finish kernel.
bool chunked_staging(const std::vector<Group> &gs, const View &vin, const View &vout, const ImgGeom &geo) {
  if (!host_one_chain(gs, vin, vout)) return false;
  void *a = nullptr, *b = nullptr;
  if (mapped_host(vin, &a) && mapped_host(vout, &b)) return false;
  return geo.rows >= 64 && vin.pitch * vin.rows >= (8 << 20);
}

mrw_status enqueue_image(Launch &L, const Program &p, const mrw_buffer *args, int nargs, const mrw_config &cfg,
                         unsigned int *status, bool *used_status) {
  View vin, vout, vred;
  TRY(validate_image_args(p, args, nargs, &vin, &vout, &vred));
  const ImgGeom geo = geom_of(args[0], vin);
  if (p.while_begin >= 0) {
    L.record = nullptr;
    return enqueue_image_while(L, p, vin, vout, geo, cfg, status, used_status);
  }
  const std::vector<Group> gs = group_stages(p, cfg.fusion == MRW_FUSE_ALL, false);
  // only a plan of one chain kernel over device buffers is replayable: nothing else is enqueued
  if (!(gs.size() == 1 && !gs[0].use_stencil && !gs[0].user && !gs[0].reduce_only &&
        vin.b->memory == MRW_MEM_DEVICE && vout.b->memory == MRW_MEM_DEVICE &&
        (p.reduce == RED_NONE || vred.b->memory == MRW_MEM_DEVICE)))
    L.record = nullptr;
  TRY(prepare_user_groups(L, gs));
  const bool one_chain = host_one_chain(gs, vin, vout);
  void *din = nullptr, *dout = nullptr;
  int64_t pin = vin.pitch, pout = vout.pitch;
  // Page-locked host buffers mapped into the device address space, read once and written once by
  // a single streaming kernel: the kernel reads and writes them in place over the host link
  // (NVLink-C2C on Grace-Blackwell), which moves the bytes faster than staging copies do.
  if (!(one_chain && mapped_host(vin, &din) && mapped_host(vout, &dout))) {
    if (L.events && chunked_staging(gs, vin, vout, geo))
      return enqueue_image_overlapped(L, gs[0], vin, vout, p.reduce != RED_NONE ? &vred : nullptr, geo, cfg, p.wg);
    TRY(resolve(L, vin, true, false, &din, &pin));
    TRY(resolve(L, vout, false, true, &dout, &pout));
  }
  unsigned long long *red = nullptr;
  void *dred = nullptr;
  int64_t pred = 0;
  if (p.reduce != RED_NONE) {
    TRY(resolve(L, vred, false, true, &dred, &pred));
    red = (unsigned long long *)dred;  // overwritten by the last CTA of the reducing launch
  }
  return run_groups(L, gs, (const uint8_t *)din, pin, (uint8_t *)dout, pout, geo, cfg, p.wg, status, used_status, red);
}

// ============================================================================================
// N-body plans
// ============================================================================================
struct NbShape {
  int grid, block, bpt;
};

// Launch shape of the force kernel: `grid` CTAs, each with 4 warp groups of T threads (each group
// sums a fixed quarter of the j range) and bpt bodies per thread, so a CTA holds T * bpt bodies.
NbShape nbody_shape(const mrw_config &cfg, int sms, int64_t n, int wg) {
  NbShape s;
  const int groups = 4;
  s.bpt = (cfg.tile_rows == 1 || cfg.tile_rows == 4) ? cfg.tile_rows : 2;
  const int cps = cfg.ctas_per_sm ? cfg.ctas_per_sm : 1;
  int64_t grid = std::min<int64_t>((int64_t)sms * cps, std::max<int64_t>(1, (n + 32 * s.bpt - 1) / (32 * s.bpt)));
  const int64_t per = (n + grid - 1) / grid;
  int64_t T = round_up((per + s.bpt - 1) / s.bpt, 32);
  if (wg && wg % (32 * groups) == 0) T = wg / groups;
  const int64_t tmax = s.bpt == 4 ? 128 : 256;  // the 4-body variant is compiled for 512 threads
  if (T > tmax) T = tmax;
  if (T * s.bpt * grid < n) grid = (n + T * s.bpt - 1) / (T * s.bpt);
  s.grid = (int)grid;
  s.block = (int)(groups * T);
  return s;
}

struct LoopGraph {
  cudaGraphExec_t exec = nullptr;
  LoopCtrl *ctrl = nullptr;
  cudaEvent_t last_use = nullptr;  // recorded behind every launch (PlanCache)
};

void destroy_loop_graph(LoopGraph &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.ctrl) cudaFree(g.ctrl);
}

PlanCache<LoopGraph> &loop_graphs() {
  static PlanCache<LoopGraph> *c = new PlanCache<LoopGraph>(64);  // never destroyed: no CUDA calls at exit
  return *c;
}

// The device-controlled Loop graph of (state arrays, constants, launch shape, stream), cached.
mrw_status get_loop_graph(const NBodyParams &np, int64_t iters, const NbShape &s, int device, cudaStream_t stream,
                          std::shared_ptr<LoopGraph> *out) {
  char key[256];
  snprintf(key, sizeof key, "%d|%p|%p|%p|%p|%d|%a|%a|%a|%lld|%d|%d|%d", device, (void *)stream, (void *)np.x,
           (void *)np.v, (void *)np.a, np.n, np.G, np.eps2, np.dt, (long long)iters, s.bpt, s.grid, s.block);
  *out = loop_graphs().find(key);
  if (*out) return MRW_OK;
  LoopGraph g;
  CU(cudaMalloc(&g.ctrl, sizeof(LoopCtrl)));
  cudaError_t e = build_nbody_loop_graph(np, g.ctrl, iters, s.bpt, s.grid, s.block, &g.exec);
  if (e != cudaSuccess) {
    cudaFree(g.ctrl);
    return cuda_fail(e, "building the Loop graph");
  }
  std::shared_ptr<LoopGraph> made;
  TRY(make_cached(g, destroy_loop_graph, &made));
  *out = loop_graphs().insert(key, made);
  return MRW_OK;
}

mrw_status validate_nbody_args(const mrw_buffer *args, int nargs, View *v) {
  if (nargs != 3) return fail(MRW_ERR_INVALID_ARG, "N-body trees take x, v, a");
  for (int i = 0; i < 3; ++i) {
    TRY(view_of(args[i], i, &v[i]));
    if (args[i].dtype != MRW_F32) return fail(MRW_ERR_DTYPE, "N-body state is float32");
    if (args[i].ndim != 2 || args[i].shape[1] != 4) return fail(MRW_ERR_SHAPE, "N-body arrays are (N, 4)");
    if (args[i].shape[0] != args[0].shape[0]) return fail(MRW_ERR_SHAPE, "x, v, a differ in N");
    if (v[i].pitch != 16) return fail(MRW_ERR_SHAPE, "N-body arrays must be dense");
    if (args[i].memory == MRW_MEM_DEVICE && (uintptr_t)args[i].data % 16)
      return fail(MRW_ERR_CONSTRAINT, "N-body arrays need 16-byte alignment");
    if (args[i].transfer != MRW_COPY && args[i].transfer != MRW_PARTITION)
      return fail(MRW_ERR_INVALID_ARG, "bad transfer mode");
  }
  if (args[0].shape[0] > INT32_MAX) return fail(MRW_ERR_SHAPE, "too many bodies");
  return MRW_OK;
}

mrw_status enqueue_nbody(Launch &L, const Program &p, const mrw_buffer *args, int nargs, const mrw_config &cfg) {
  View v[3];
  TRY(validate_nbody_args(args, nargs, v));
  const int64_t n = args[0].shape[0];
  void *d[3];
  int64_t pitch;
  for (int i = 0; i < 3; ++i) TRY(resolve(L, v[i], true, true, &d[i], &pitch));
  NBodyParams np;
  np.x = (float4 *)d[0];
  np.v = (float4 *)d[1];
  np.a = (float4 *)d[2];
  np.n = (int32_t)n;
  const NbShape s = nbody_shape(cfg, L.sms, n, p.wg);
  for (const NbStep &st : p.nb) {
    np.G = st.G > 0.f ? st.G : (float)(1.0 / (double)n);
    np.eps2 = st.eps * st.eps;
    np.dt = st.dt;
    if (st.accel) {
      CU(launch_nbody_force(np, 0, s.bpt, s.grid, s.block, L.stream));
      continue;
    }
    if (cfg.fusion == MRW_FUSE_NONE) {
      // kernel per step and host-evaluated loop condition (the paper's Loop, Section 3.1)
      for (int64_t it = 0; it < st.iters; ++it) {
        CU(launch_nbody_drift(np, L.stream));
        CU(launch_nbody_force(np, 0, s.bpt, s.grid, s.block, L.stream));
        CU(launch_nbody_kick(np, L.stream));
        if (st.from_loop) CU(cudaStreamSynchronize(L.stream));
      }
    } else if (st.from_loop) {
      std::shared_ptr<LoopGraph> g;
      TRY(get_loop_graph(np, st.iters, s, L.device, L.stream, &g));
      RecordOnExit used_until{g->last_use, L.stream};
      CU(cudaGraphLaunch(g->exec, L.stream));
    } else {
      for (int64_t it = 0; it < st.iters; ++it) {
        CU(launch_nbody_drift(np, L.stream));
        CU(launch_nbody_force(np, 1, s.bpt, s.grid, s.block, L.stream));
      }
    }
  }
  return MRW_OK;
}

// ============================================================================================
// Saxpy
// ============================================================================================
mrw_status validate_saxpy_args(const mrw_buffer *args, int nargs, View *vx, View *vy) {
  if (nargs != 2) return fail(MRW_ERR_INVALID_ARG, "saxpy takes x, y");
  TRY(view_of(args[0], 0, vx));
  TRY(view_of(args[1], 1, vy));
  if (args[0].dtype != MRW_F32 || args[1].dtype != MRW_F32) return fail(MRW_ERR_DTYPE, "saxpy is float32");
  if (vx->numel() != vy->numel()) return fail(MRW_ERR_SHAPE, "x and y differ in size");
  if (vx->pitch != vx->width * 4 || vy->pitch != vy->width * 4) return fail(MRW_ERR_SHAPE, "saxpy vectors must be dense");
  for (int i = 0; i < 2; ++i)
    if (args[i].memory == MRW_MEM_DEVICE && (uintptr_t)args[i].data % 16)
      return fail(MRW_ERR_CONSTRAINT, "saxpy vectors need 16-byte alignment");
  return MRW_OK;
}

mrw_status enqueue_saxpy(Launch &L, const Program &p, const mrw_buffer *args, int nargs, const mrw_config &cfg) {
  View vx, vy;
  TRY(validate_saxpy_args(args, nargs, &vx, &vy));
  void *dx, *dy;
  int64_t pp;
  TRY(resolve(L, vx, true, false, &dx, &pp));
  TRY(resolve(L, vy, true, true, &dy, &pp));
  if (p.wg && p.wg != 256) return fail(MRW_ERR_UNSUPPORTED, "saxpy runs in CTAs of 256 threads");
  // FUSE_ALL: consecutive stages fused, up to kMaxSaxpyStages per pass over the vectors;
  // FUSE_NONE: one pass per stage (the kernel-per-stage baseline). unroll: float4 groups per thread.
  SaxpyArgs a{};
  a.x = (const float *)dx;
  a.y = (float *)dy;
  a.n = vx.numel();
  const int unroll = cfg.unroll ? cfg.unroll : 4;
  const size_t per = cfg.fusion == MRW_FUSE_ALL ? (size_t)kMaxSaxpyStages : 1;
  for (size_t s0 = 0; s0 < p.alphas.size(); s0 += per) {
    a.nstages = (int32_t)std::min(per, p.alphas.size() - s0);
    for (int k = 0; k < a.nstages; ++k) a.alpha[k] = p.alphas[s0 + k];
    CU(launch_saxpy(a, unroll, L.stream));
  }
  return MRW_OK;
}

// ============================================================================================
// Knowledge base (Section 3.2: profiles of past executions)
// ============================================================================================
struct KbRecord {
  mrw_config cfg;
  float ms;
  int source;  // 0 exhaustive, 1 pruned, 2 model
};
std::map<std::string, KbRecord> &kb() {
  static std::map<std::string, KbRecord> m;
  return m;
}

std::string workload_signature(const mrw_buffer *args, int nargs) {
  std::string s;
  char buf[128];
  for (int i = 0; i < nargs; ++i) {
    snprintf(buf, sizeof buf, "%d:%d:", (int)args[i].dtype, args[i].ndim);
    s += buf;
    for (int d = 0; d < args[i].ndim && d < MRW_MAX_DIMS; ++d) {
      snprintf(buf, sizeof buf, "%lldx", (long long)args[i].shape[d]);
      s += buf;
    }
    snprintf(buf, sizeof buf, "p%lld;", (long long)args[i].pitch);
    s += buf;
  }
  return s;
}

std::string tree_signature(const mrw_node *n) {
  std::string s;
  signature(n, s);
  return s;
}

struct ModelSlot {
  mrw_model *model = nullptr;
  std::vector<mrw_config> cfgs;
};
ModelSlot &installed_model() {
  static ModelSlot m;
  return m;
}

}  // namespace

// ============================================================================================
// Cost model object
// ============================================================================================
struct mrw_model {
  MlpDims d{};
  int device = 0;
  float *master = nullptr, *m = nullptr, *v = nullptr, *grads = nullptr, *loss = nullptr;
  uint16_t *bf = nullptr;
  int32_t *idx = nullptr;
  int64_t idx_cap = 0;
  int64_t step = 0;
};

namespace {

mrw_status get_program(const mrw_node *root, Program *p) {
  if (!root) return fail(MRW_ERR_INVALID_ARG, "root is NULL");
  TRY(flatten(root, *p, 0, true, 1));
  if (p->fam == F_NONE) return fail(MRW_ERR_INVALID_ARG, "the tree has no stages");
  if (p->while_begin >= 0 && p->reduce != RED_NONE)
    return fail(MRW_ERR_UNSUPPORTED, "a WHILE_CHANGED loop inside a MapReduce");
  return MRW_OK;
}

mrw_status model_predict(mrw_model *m, const float *feat, int *best);
mrw_status features_of(const Program &p, const mrw_buffer *args, int nargs, float *f);

// ============================================================================================
// FFT trees: rows of kFftN complex values; up to kFftMaxSteps transforms per cluster launch
// ============================================================================================
mrw_status validate_fft_args(const mrw_buffer *args, int nargs, View *vx, View *vy) {
  if (nargs != 2) return fail(MRW_ERR_INVALID_ARG, "FFT trees take x, y");
  TRY(view_of(args[0], 0, vx));
  TRY(view_of(args[1], 1, vy));
  if (args[0].dtype != MRW_C64 || args[1].dtype != MRW_C64)
    return fail(MRW_ERR_DTYPE, "FFT stages read and write complex float32 (MRW_C64)");
  if (!same_shape(args[0], args[1])) return fail(MRW_ERR_SHAPE, "x and y differ in shape");
  if (vx->width != kFftN) return fail(MRW_ERR_SHAPE, "FFT rows hold %d values, not %lld", kFftN, (long long)vx->width);
  for (int i = 0; i < 2; ++i) {
    const View &v = i ? *vy : *vx;
    if (v.pitch != (int64_t)kFftN * 8) return fail(MRW_ERR_SHAPE, "args[%d]: FFT rows must be dense", i);
    if (v.b->memory == MRW_MEM_DEVICE && (uintptr_t)v.b->data % 16)
      return fail(MRW_ERR_CONSTRAINT, "args[%d]: FFT rows need a 16-byte aligned pointer", i);
  }
  if (args[0].memory == MRW_MEM_DEVICE && args[1].memory == MRW_MEM_DEVICE) {
    const uintptr_t a0 = (uintptr_t)args[0].data, a1 = a0 + vx->pitch * vx->rows;
    const uintptr_t b0 = (uintptr_t)args[1].data, b1 = b0 + vy->pitch * vy->rows;
    if (a0 != b0 && a0 < b1 && b0 < a1) return fail(MRW_ERR_INVALID_ARG, "y overlaps x without being x");
  }
  return MRW_OK;
}

// Which FFT kernel runs the rows. Clusters of 8 CTAs keep a row on chip, the exchange's values in
// registers (two CTAs per SM; 36 clusters at once on GB300) or in TMEM (three per SM; 51
// clusters); the L2-ring form splits each row's phases into work items of a persistent grid and
// exchanges the values through an L2-resident ring. Every row of a cluster form runs at once up to
// the clusters' residency, and there the forms are within a few microseconds of each other (the
// register form ahead at 4-12 rows and for single transforms, the ring form for pairs of 16-36
// rows); beyond it the L2-ring form is the fastest measured (41 us for a forward and inverse pair
// of 64 rows, 125 at 256, 236 at 512, against 48, 174 and 340 for the TMEM form). The default takes
// the L2-ring form exactly when nfft exceeds the register form's residency. cfg.ctas_per_sm 1 asks
// for the L2-ring form, 2 for the register form, 4 for the TMEM form and 3 for clusters of 16 CTAs
// (three per SM, where the device allows that cluster size).
enum FftForm { FFT_REG, FFT_TMEM, FFT_C16, FFT_L2 };
FftForm fft_form(const mrw_config &cfg, int64_t nfft) {
  if (cfg.ctas_per_sm == 1 && fft_l2_ctas_per_sm() > 0) return FFT_L2;
  if (cfg.ctas_per_sm == 3 && fft16_max_clusters() > 0) return FFT_C16;
  if (cfg.ctas_per_sm == 2) return FFT_REG;
  const int tm = fft_max_clusters(true), reg = fft_max_clusters(false);
  if (cfg.ctas_per_sm == 4) return tm > 0 ? FFT_TMEM : FFT_REG;
  if (nfft > reg && fft_l2_ctas_per_sm() > 0) return FFT_L2;
  return tm > reg && nfft > reg ? FFT_TMEM : FFT_REG;
}

// The L2-ring form: one workspace (the ring and the completion counters, sized for the largest
// launch) serves every launch of the chain in stream order.
mrw_status enqueue_fft_l2(Launch &L, const Program &p, const float2 *dx, float2 *dy, int64_t nfft, int per,
                          unsigned int *status, bool *used_status) {
  const int ctas = fft_l2_ctas_per_sm() * L.sms;
  std::vector<FftL2Plan> plans;
  size_t ring = 0, counters = 0;
  for (size_t i = 0; i < p.fft.size(); i += per) {
    FftL2Plan pl{};
    if (!fft_l2_plan(nfft, (int)std::min<size_t>(per, p.fft.size() - i), ctas, &pl))
      return fail(MRW_ERR_UNSUPPORTED, "%lld FFT rows do not fit the L2-ring schedule", (long long)nfft);
    ring = std::max(ring, pl.ring_bytes);
    counters = std::max(counters, pl.counter_bytes);
    plans.push_back(pl);
  }
  void *ws = nullptr;
  const size_t ring_padded = (ring + 255) / 256 * 256;
  TRY(L.alloc(&ws, ring_padded + counters));
  FftL2Args a{};
  a.in = dx;
  a.out = dy;
  a.ring = (float2 *)ws;
  a.done = (unsigned int *)((char *)ws + ring_padded);
  a.status = status;
  a.wait_polls = test_wait_polls();
  CU(fft_l2_twiddles(&a.twiddle));
  if (status) *used_status = true;
  for (size_t i = 0, c = 0; i < p.fft.size(); i += per, ++c) {
    const FftL2Plan &pl = plans[c];
    a.sc = pl.sc;
    a.ring_rows = pl.ring_rows;
    a.ticket = a.done + pl.sc.nfft * pl.sc.P;
    a.nsteps = pl.sc.P - 1;
    for (int k = 0; k < a.nsteps; ++k) a.sign[k] = p.fft[i + k];
    CU(launch_fft_l2(a, pl.ctas, L.stream));
    a.in = dy;  // later launches continue in place on y
  }
  return MRW_OK;
}

mrw_status enqueue_fft(Launch &L, const Program &p, const mrw_buffer *args, int nargs, const mrw_config &cfg,
                       unsigned int *status, bool *used_status) {
  View vx, vy;
  TRY(validate_fft_args(args, nargs, &vx, &vy));
  const bool inplace = args[0].data == args[1].data;
  void *dx, *dy;
  int64_t pp;
  TRY(resolve(L, vx, true, inplace, &dx, &pp));
  if (inplace) {
    dy = dx;
  } else {
    TRY(resolve(L, vy, false, true, &dy, &pp));
  }
  const FftForm form = fft_form(cfg, vx.rows);
  const int per = cfg.fusion == MRW_FUSE_ALL ? kFftMaxSteps : 1;
  if (form == FFT_L2) return enqueue_fft_l2(L, p, (const float2 *)dx, (float2 *)dy, vx.rows, per, status, used_status);
  const bool tm = form == FFT_TMEM;
  const int max16 = form == FFT_C16 ? fft16_max_clusters() : 0;
  const int maxc = max16 > 0 ? max16 : fft_max_clusters(tm);
  if (maxc < 1) return fail(MRW_ERR_UNSUPPORTED, "a %d-CTA cluster with %zu bytes of shared memory does not fit",
                            kFftCluster, fft_smem_bytes());
  FftArgs a{};
  a.nfft = vx.rows;
  a.status = max16 > 0 ? status : nullptr;
  if (a.status) *used_status = true;
  const int clusters = (int)std::min<int64_t>(a.nfft, maxc);
  a.in = (const float2 *)dx;
  a.out = (float2 *)dy;
  for (size_t i = 0; i < p.fft.size(); i += per) {
    a.nsteps = (int32_t)std::min<size_t>(per, p.fft.size() - i);
    for (int k = 0; k < a.nsteps; ++k) a.sign[k] = p.fft[i + k];
    if (max16 > 0) CU(launch_fft16(a, clusters, L.stream));
    else CU(launch_fft(a, clusters, tm, L.stream));
    a.in = (const float2 *)dy;  // later launches continue in place on y
  }
  return MRW_OK;
}

// Argument checks of every family, before any CUDA call.
mrw_status validate_args(const Program &p, const mrw_buffer *args, int nargs) {
  if (nargs < 0 || (nargs && !args)) return fail(MRW_ERR_INVALID_ARG, "bad argument list");
  if (p.fam == F_IMAGE) {
    View a, b, c;
    return validate_image_args(p, args, nargs, &a, &b, &c);
  }
  if (p.fam == F_NBODY) {
    View v[3];
    return validate_nbody_args(args, nargs, v);
  }
  View x, y;
  if (p.fam == F_FFT) return validate_fft_args(args, nargs, &x, &y);
  return validate_saxpy_args(args, nargs, &x, &y);
}

// Configuration for an execution without an explicit one: knowledge base, then the cost model
// (recorded in the knowledge base as derived), then the default (Section 3.2, Fig. 4 decision).
mrw_config pick_config(const mrw_node *root, const Program &p, const mrw_buffer *args, int nargs) {
  const std::string key = tree_signature(root) + "|" + workload_signature(args, nargs);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = kb().find(key);
    if (it != kb().end()) return it->second.cfg;
  }
  mrw_model *m = nullptr;
  std::vector<mrw_config> cfgs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    m = installed_model().model;
    cfgs = installed_model().cfgs;
  }
  if (m && (int)cfgs.size() == m->d.k) {
    float f[MRW_NFEATURES];
    int best = -1;
    if (features_of(p, args, nargs, f) == MRW_OK && model_predict(m, f, &best) == MRW_OK && best >= 0) {
      std::lock_guard<std::mutex> lk(g_mu);
      kb()[key] = {cfgs[best], -1.f, 2};
      bump_plan_gen();
      return cfgs[best];
    }
  }
  return default_config(p.fam);
}

// Enqueue one execution (no future); shared by mrw_execute and the tuner.
mrw_status enqueue(Launch &L, const Program &p, const mrw_buffer *args, int nargs, const mrw_config &cfg,
                   unsigned int *status, bool *used_status) {
  TRY(check_config(cfg));
  switch (p.fam) {
    case F_IMAGE: TRY(enqueue_image(L, p, args, nargs, cfg, status, used_status)); break;
    case F_NBODY: TRY(enqueue_nbody(L, p, args, nargs, cfg)); break;
    case F_SAXPY: TRY(enqueue_saxpy(L, p, args, nargs, cfg)); break;
    case F_FFT: TRY(enqueue_fft(L, p, args, nargs, cfg, status, used_status)); break;
    default: return fail(MRW_ERR_INVALID_ARG, "empty tree");
  }
  TRY(copy_back(L));
  return MRW_OK;
}

mrw_status begin_launch(Launch &L, void *stream) {
  L.stream = (cudaStream_t)stream;
  CU(cudaGetDevice(&L.device));
  L.sms = device_info(L.device).sms;
  configure_pool(L.device);
  return MRW_OK;
}

// The future's completion event: an ordering-only event, or a timing pair when asked for.
mrw_status take_future_events(mrw_future *f, bool timed) {
  f->timed = timed;
  if (timed) return event_pool().take(&f->start, &f->done);
  return get_sync_event(&f->done);
}

void free_future(mrw_future *f) {
  if (!f) return;
  if (f->timed) {
    event_pool().give(f->start, f->done);
  } else if (f->done) {
    f->sync_events.push_back(f->done);
  }
  put_sync_events(f->sync_events);
  status_pool().give(f->slot);
  result_pool().give(f->result_slot);
  delete f;
}

}  // namespace

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

int32_t mrw_abi_version(void) { return MRW_ABI_VERSION; }

const char *mrw_last_error(void) { return t_err.c_str(); }

const char *mrw_status_string(mrw_status s) {
  switch (s) {
    case MRW_OK: return "ok";
    case MRW_ERR_INVALID_ARG: return "invalid argument";
    case MRW_ERR_SHAPE: return "shape mismatch";
    case MRW_ERR_DTYPE: return "dtype mismatch";
    case MRW_ERR_CONSTRAINT: return "partitioning constraint violated";
    case MRW_ERR_OOM: return "out of memory";
    case MRW_ERR_CUDA: return "CUDA error";
    case MRW_ERR_TIMEOUT: return "timeout";
    case MRW_ERR_DEVICE: return "device-side error";
    case MRW_ERR_UNSUPPORTED: return "unsupported";
    case MRW_ERR_NOT_READY: return "not ready";
  }
  return "unknown status";
}

mrw_status mrw_stage(mrw_stage_kind kind, const mrw_stage_params *params, mrw_node_t *out) {
  if (!out) return fail(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!valid_stage_kind(kind)) return fail(MRW_ERR_INVALID_ARG, "unknown stage kind %d", (int)kind);
  mrw_node *n = new_node(N_STAGE);
  if (!n) return fail(MRW_ERR_OOM, "node");
  n->stage = kind;
  n->params = default_params(kind, params);
  *out = n;
  return MRW_OK;
}

mrw_status mrw_stage_user(const char *name, const char *source, const uint32_t *params, mrw_node_t *out) {
  if (!out) return fail(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!name || !source || !*name || !*source) return fail(MRW_ERR_INVALID_ARG, "name and source must be non-empty");
  const size_t nl = strlen(name);
  bool ident = nl <= 63 && (isalpha((unsigned char)name[0]) || name[0] == '_');
  for (size_t i = 1; ident && i < nl; ++i) ident = isalnum((unsigned char)name[i]) || name[i] == '_';
  if (!ident) return fail(MRW_ERR_INVALID_ARG, "stage name must be a C identifier of at most 63 characters");
  if (strlen(source) > (64u << 10)) return fail(MRW_ERR_INVALID_ARG, "user stage source above 64 KiB");
  auto fn = std::make_shared<mrw_user_fn>();
  fn->name = name;
  fn->source = source;
  // compile the function once inside a one-stage group, for the current device's architecture
  // (sm_103 when no device is visible), so that errors surface here and not at execution
  int dev = 0, arch = 103;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    const int a = device_info(dev).arch;
    if (a > 0) arch = a;
  } else {
    cudaGetLastError();
  }
  Group g;
  g.user = true;
  ImgStage st{OP_USER, 0, 0, 0, 0};
  st.fn = fn;
  g.pre.push_back(st);
  std::string err;
  if (!jit_check(user_chain_source(g), arch, &err)) return fail(MRW_ERR_UNSUPPORTED, "%s", err.c_str());
  mrw_node *n = new_node(N_STAGE);
  if (!n) return fail(MRW_ERR_OOM, "node");
  n->user = fn;
  if (params) std::copy(params, params + kUserParams, n->uparams);
  *out = n;
  return MRW_OK;
}

mrw_status mrw_pipeline_create(mrw_node_t *out) {
  if (!out) return fail(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = new_node(N_PIPELINE);
  return *out ? MRW_OK : fail(MRW_ERR_OOM, "node");
}

mrw_status mrw_pipeline_add_node(mrw_node_t pipe, mrw_node_t child) {
  if (!pipe || !child) return fail(MRW_ERR_INVALID_ARG, "NULL node");
  if (pipe->kind != N_PIPELINE) return fail(MRW_ERR_INVALID_ARG, "not a pipeline");
  if (contains(child, pipe)) return fail(MRW_ERR_INVALID_ARG, "adding a node to its own subtree");
  child->refs.fetch_add(1);
  pipe->kids.push_back(child);
  bump_plan_gen();
  return MRW_OK;
}

mrw_status mrw_pipeline_add_stage(mrw_node_t pipe, mrw_stage_kind kind, const mrw_stage_params *params) {
  if (!pipe) return fail(MRW_ERR_INVALID_ARG, "NULL pipeline");
  if (pipe->kind != N_PIPELINE) return fail(MRW_ERR_INVALID_ARG, "not a pipeline");
  mrw_node_t st;
  TRY(mrw_stage(kind, params, &st));
  pipe->kids.push_back(st);  // the pipeline takes over the creation reference
  bump_plan_gen();
  return MRW_OK;
}

static mrw_status wrap(NodeKind k, mrw_node_t body, mrw_node_t *out) {
  if (!out) return fail(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!body) return fail(MRW_ERR_INVALID_ARG, "body is NULL");
  mrw_node *n = new_node(k);
  if (!n) return fail(MRW_ERR_OOM, "node");
  body->refs.fetch_add(1);
  n->kids.push_back(body);
  *out = n;
  return MRW_OK;
}

mrw_status mrw_map(mrw_node_t body, mrw_node_t *out) { return wrap(N_MAP, body, out); }

mrw_status mrw_mapreduce(mrw_node_t map_body, mrw_reduce_op op, mrw_node_t *out) {
  if (op < MRW_RED_ADD || op > MRW_RED_DIV) return fail(MRW_ERR_INVALID_ARG, "unknown merging function");
  TRY(wrap(N_MAPREDUCE, map_body, out));
  (*out)->op = op;
  return MRW_OK;
}

mrw_status mrw_loop(mrw_node_t body, const mrw_loop_state *state, mrw_node_t *out) {
  if (!state) return fail(MRW_ERR_INVALID_ARG, "state is NULL");
  if (state->max_iters < 0 || state->max_iters > 100000000) return fail(MRW_ERR_INVALID_ARG, "max_iters out of range");
  if (state->kind != MRW_LOOP_FOR && state->kind != MRW_LOOP_WHILE_CHANGED)
    return fail(MRW_ERR_UNSUPPORTED, "loop kind %d", state->kind);
  TRY(wrap(N_LOOP, body, out));
  (*out)->loop = *state;
  return MRW_OK;
}

void mrw_node_retain(mrw_node_t n) {
  if (n) n->refs.fetch_add(1);
}

void mrw_node_release(mrw_node_t n) { release_node(n); }

}  // extern "C"

namespace {
thread_local ChainReplay t_replay;  // the last replayable launch of this thread

bool replay_matches(const ChainReplay &r, const mrw_node *root, const mrw_buffer *args, int32_t nargs,
                    const mrw_config *cfg, cudaStream_t stream, int device) {
  return r.valid && r.root == root && r.nargs == nargs && r.stream == stream && r.device == device &&
         r.gen == g_plan_gen.load(std::memory_order_acquire) && r.has_cfg == (cfg != nullptr) &&
         (!cfg || memcmp(&r.cfg, cfg, sizeof(mrw_config)) == 0) &&
         memcmp(r.args, args, (size_t)nargs * sizeof(mrw_buffer)) == 0;
}

mrw_status replay_chain(const ChainReplay &r, bool timed, mrw_future_t *out) {
  mrw_future *f = new (std::nothrow) mrw_future();
  if (!f) return fail(MRW_ERR_OOM, "future");
  f->device = r.device;
  mrw_status s = take_future_events(f, timed);
  if (s != MRW_OK) {
    free_future(f);
    return s;
  }
  if (r.finish_nout > 0) {  // a MapReduce: the result is in the call's args[2] (device memory)
    f->nresult = r.finish_nout;
    f->result_src = r.args[2].data;
    f->result_mem = r.args[2].memory;
  }
  if (timed) cudaEventRecord(f->start, r.stream);
  cudaError_t e;
  if (r.finish_nout > 0) {
    std::lock_guard<std::mutex> lk(g_reduce_mu);
    e = launch_chain(r.a, r.n_noise, r.unroll, r.grid, r.block, r.stream);
    if (e == cudaSuccess) e = launch_chain_finish(r.a.partials, r.a.red, r.finish_nout, r.stream);
  } else {
    e = launch_chain(r.a, r.n_noise, r.unroll, r.grid, r.block, r.stream);
  }
  cudaEventRecord(f->done, r.stream);
  if (e != cudaSuccess) {
    const mrw_status st = cuda_fail(e, "chain kernel launch");
    const std::string msg = t_err;
    cudaEventSynchronize(f->done);
    free_future(f);
    t_err = msg;
    return st;
  }
  *out = f;
  return MRW_OK;
}

mrw_status execute(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfg, void *stream,
                   mrw_future_t *out, bool timed) {
  if (!out) return fail(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nargs < 0 || (nargs && !args)) return fail(MRW_ERR_INVALID_ARG, "bad argument list");
  const bool replayable = root && nargs >= 2 && nargs <= 3;
  if (replayable && t_replay.valid) {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        replay_matches(t_replay, root, args, nargs, cfg, (cudaStream_t)stream, dev))
      return replay_chain(t_replay, timed, out);
  }
  const uint64_t gen = g_plan_gen.load(std::memory_order_acquire);  // before anything is planned
  Program p;
  TRY(get_program(root, &p));
  // A MapReduce called without a result buffer: the future owns the result, in a page-locked slot
  // that the call's work fills (the slot is a host args[2], staged like any host buffer).
  struct SlotGuard {
    int64_t *p = nullptr;
    ~SlotGuard() { result_pool().give(p); }
  } own_slot;
  mrw_buffer own[3];
  if (p.fam == F_IMAGE && p.reduce != RED_NONE && nargs == 2) {
    TRY(result_pool().take(&own_slot.p));
    own[0] = args[0];
    own[1] = args[1];
    own[2] = mrw_buffer{};
    own[2].data = own_slot.p;
    own[2].dtype = MRW_I64;
    own[2].ndim = 1;
    own[2].shape[0] = p.reduce == RED_COUNT3 ? 3 : 1;
    own[2].memory = MRW_MEM_HOST;
    args = own;
    nargs = 3;
  }
  TRY(validate_args(p, args, nargs));
  const mrw_config c = cfg ? *cfg : pick_config(root, p, args, nargs);
  TRY(check_config(c));
  Launch L;
  TRY(begin_launch(L, stream));
  mrw_future *f = new (std::nothrow) mrw_future();
  if (!f) return fail(MRW_ERR_OOM, "future");
  f->device = L.device;
  mrw_status s = status_pool().take(&f->slot);
  if (s == MRW_OK) s = take_future_events(f, timed);
  if (s != MRW_OK) {
    free_future(f);
    return s;
  }
  if (p.fam == F_IMAGE && p.reduce != RED_NONE) {
    f->nresult = p.reduce == RED_COUNT3 ? 3 : 1;
    if (own_slot.p) {
      f->result_slot = own_slot.p;
      own_slot.p = nullptr;
    } else {
      f->result_src = args[2].data;
      f->result_mem = args[2].memory;
    }
  }
  if (timed) cudaEventRecord(f->start, L.stream);
  bool used = false;
  L.events = &f->sync_events;
  ChainReplay rec;
  L.record = replayable && p.fam == F_IMAGE ? &rec : nullptr;
  s = enqueue(L, p, args, nargs, c, f->slot.dev, &used);
  f->has_status = used;  // kernels write failures into the mapped host word itself
  L.free_all();
  cudaEventRecord(f->done, L.stream);
  if (s == MRW_OK && L.record && L.recorded && !used) {
    rec.valid = true;
    rec.gen = gen;
    rec.root = root;
    rec.device = L.device;
    rec.stream = L.stream;
    rec.nargs = nargs;
    memcpy(rec.args, args, (size_t)nargs * sizeof(mrw_buffer));
    rec.has_cfg = cfg != nullptr;
    if (cfg) rec.cfg = *cfg;
    t_replay = rec;
  }
  if (s != MRW_OK) {
    // what was enqueued still runs; wait for it so the future's resources can go
    const std::string msg = t_err;
    cudaEventSynchronize(f->done);
    free_future(f);
    t_err = msg;
    return s;
  }
  *out = f;
  return MRW_OK;
}
}  // namespace

extern "C" {

mrw_status mrw_execute(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfg, void *stream,
                       mrw_future_t *out) {
  return execute(root, args, nargs, cfg, stream, out, false);
}

mrw_status mrw_execute_timed(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfg,
                             void *stream, mrw_future_t *out) {
  return execute(root, args, nargs, cfg, stream, out, true);
}

mrw_status mrw_future_query(mrw_future_t f) {
  if (!f) return fail(MRW_ERR_INVALID_ARG, "future is NULL");
  const cudaError_t e = cudaEventQuery(f->done);
  if (e == cudaErrorNotReady) return MRW_ERR_NOT_READY;
  if (e != cudaSuccess) return cuda_fail(e, "stream of the future");
  if (f->has_status && *(volatile unsigned int *)f->slot.host != 0)
    return fail(MRW_ERR_DEVICE, "a kernel gave up a bounded wait (status %u)", *f->slot.host);
  return f->deferred;
}

mrw_status mrw_future_wait(mrw_future_t f, int64_t timeout_ms) {
  if (!f) return fail(MRW_ERR_INVALID_ARG, "future is NULL");
  if (timeout_ms < 0) {
    const cudaError_t e = cudaEventSynchronize(f->done);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    return mrw_future_query(f);
  }
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    const mrw_status s = mrw_future_query(f);
    if (s != MRW_ERR_NOT_READY) return s;
    const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
    if (el.count() >= timeout_ms) return fail(MRW_ERR_TIMEOUT, "future not complete after %lld ms", (long long)timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

mrw_status mrw_future_elapsed_ms(mrw_future_t f, float *ms) {
  if (!f || !ms) return fail(MRW_ERR_INVALID_ARG, "NULL argument");
  if (!f->timed) return fail(MRW_ERR_INVALID_ARG, "the future records no time: run with mrw_execute_timed");
  const cudaError_t e = cudaEventElapsedTime(ms, f->start, f->done);
  if (e == cudaErrorNotReady) return MRW_ERR_NOT_READY;
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
  return MRW_OK;
}

mrw_status mrw_future_result(mrw_future_t f, void *host_dst, size_t bytes) {
  if (!f || !host_dst) return fail(MRW_ERR_INVALID_ARG, "NULL argument");
  if (f->nresult == 0) return fail(MRW_ERR_INVALID_ARG, "the executed tree has no reduction: the future carries no result");
  const size_t need = (size_t)f->nresult * sizeof(int64_t);
  if (bytes < need) return fail(MRW_ERR_INVALID_ARG, "the result takes %zu bytes, the destination has %zu", need, bytes);
  TRY(mrw_future_wait(f, -1));
  if (f->result_slot) {
    memcpy(host_dst, f->result_slot, need);
  } else if (f->result_mem == MRW_MEM_HOST) {
    memcpy(host_dst, f->result_src, need);
  } else {
    // the call's work has completed, so a copy on a private stream of the future's device reads
    // the final values; the caller's device is restored afterwards
    int prev = -1;
    CU(cudaGetDevice(&prev));
    if (prev != f->device) CU(cudaSetDevice(f->device));
    cudaStream_t rs = nullptr;
    mrw_status st = result_stream(f->device, &rs);
    cudaError_t e = cudaSuccess;
    if (st == MRW_OK) {
      std::lock_guard<std::mutex> lk(g_result_mu);
      e = cudaMemcpyAsync(host_dst, f->result_src, need, cudaMemcpyDeviceToHost, rs);
      if (e == cudaSuccess) e = cudaStreamSynchronize(rs);
    }
    if (prev != f->device) cudaSetDevice(prev);
    TRY(st);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the MapReduce result");
  }
  return MRW_OK;
}

void mrw_future_release(mrw_future_t f) {
  if (!f) return;
  cudaEventSynchronize(f->done);  // the status slot must not be reused while a copy is pending
  free_future(f);
}

// --------------------------------------------------------------------------------------------
// Batched execution (pattern: thousands of uneven instances of one tree in one launch)
// --------------------------------------------------------------------------------------------
}  // extern "C"

namespace {

struct BatchPlan {
  std::vector<void *> owned;      // device tables (cudaMalloc)
  void *tmp_arena[2] = {nullptr, nullptr};
  unsigned int *counters = nullptr;  // one queue counter per group + a status word
  cudaGraphExec_t exec = nullptr;
  int ngroups = 0;
  cudaEvent_t last_use = nullptr;  // recorded behind every launch (PlanCache)
};

PlanCache<BatchPlan> &batch_plans() {
  static PlanCache<BatchPlan> *c = new PlanCache<BatchPlan>(32);  // never destroyed: no CUDA calls at exit
  return *c;
}

void destroy_batch_plan(BatchPlan &b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  for (void *p : b.owned) cudaFree(p);
  if (b.tmp_arena[0]) cudaFree(b.tmp_arena[0]);
  if (b.tmp_arena[1]) cudaFree(b.tmp_arena[1]);
  if (b.counters) cudaFree(b.counters);
}

uint64_t hash_bytes(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
  const uint8_t *b = (const uint8_t *)p;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

mrw_status build_batch_plan(Launch &L, const Program &p, const uint8_t *in_arena, uint8_t *out_arena,
                            int64_t arena_bytes, const int64_t *desc, int64_t n, const mrw_config &cfg,
                            BatchPlan *bp) {
  const std::vector<Group> gs = group_stages(p, cfg.fusion == MRW_FUSE_ALL, true);
  bp->ngroups = (int)gs.size();
  CU(cudaMalloc(&bp->counters, sizeof(unsigned int) * (gs.size() + 1)));
  if (gs.size() > 1) CU(cudaMalloc(&bp->tmp_arena[0], (size_t)arena_bytes));
  if (gs.size() > 2) CU(cudaMalloc(&bp->tmp_arena[1], (size_t)arena_bytes));
  CU(stencil_prepare());
  cudaStream_t cs;
  CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  Launch C = L;
  C.stream = cs;
  std::vector<StencilArgs> launches;
  std::vector<int> grids, blocks;
  std::vector<size_t> smems;
  // Instances in decreasing order of pixels, so the persistent workers take the largest first and
  // the end of the launch is made of small items (longest-first scheduling of the tile queue).
  std::vector<int64_t> order((size_t)n);
  for (int64_t i = 0; i < n; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    return desc[5 * x + 1] * desc[5 * x + 2] > desc[5 * y + 1] * desc[5 * y + 2];
  });
  const uint8_t *src = in_arena;
  for (size_t gi = 0; gi < gs.size(); ++gi) {
    const Group &g = gs[gi];
    StencilArgs a{};
    fill_stencil_ops(g, a);
    const StencilShape s = stencil_shape(cfg, a);
    uint8_t *dst = gi + 1 == gs.size() ? out_arena : (uint8_t *)bp->tmp_arena[gi & 1];
    StencilTables t;
    t.maps.resize((size_t)n);
    t.inst.resize((size_t)n);
    t.prefix.resize((size_t)n + 1);
    int64_t tiles = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t d = order[(size_t)i];
      const int64_t off = desc[5 * d], W = desc[5 * d + 1], H = desc[5 * d + 2], pitch = desc[5 * d + 3];
      const cudaError_t e = encode_u8_map(&t.maps[i], src + off, W, H, 1, pitch, s.box_w, s.box_h);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(e, "encoding a tensor map");
      }
      StencilInstance &in = t.inst[i];
      in.in_off = off;
      in.out_off = off;
      in.W = (int32_t)W;
      in.H = (int32_t)H;
      in.D = 1;
      in.pitch_in = in.pitch_out = (int32_t)pitch;
      in.seed_xor = (uint32_t)desc[5 * d + 4];
      in.tiles_x = (int32_t)((W + s.tile_w - 1) / s.tile_w);
      in.tiles_y = (int32_t)((H + s.tile_h - 1) / s.tile_h);
      in.tile_base = tiles;
      t.prefix[i] = tiles;
      tiles += (int64_t)in.tiles_x * in.tiles_y;
    }
    t.prefix[n] = tiles;
    t.total = tiles;
    if (tiles >= (int64_t)1 << 31) {
      cudaStreamDestroy(cs);
      return fail(MRW_ERR_UNSUPPORTED, "too many tiles in one batch");
    }
    void *dm, *di, *dp;
    mrw_status st = upload_tables(C, t, &dm, &di, &dp, true, &bp->owned);
    if (st != MRW_OK) {
      cudaStreamDestroy(cs);
      return st;
    }
    a.maps = (const CUtensorMap *)dm;
    a.inst = (const StencilInstance *)di;
    a.tile_prefix = (const int64_t *)dp;
    a.in_base = src;
    a.out_base = dst;
    a.queue = bp->counters + gi;
    a.status = bp->counters + gs.size();
    a.total_tiles = tiles;
    a.ninst = (int32_t)n;
    apply_shape(a, s);
    launches.push_back(a);
    grids.push_back(stencil_grid(s, a, tiles, L.sms));
    blocks.push_back(s.block);
    smems.push_back(s.smem);
    src = dst;
  }
  // one graph, built node by node: reset the counters, then the persistent launches
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  NodeChain nc;
  nc.g = graph;
  if (e == cudaSuccess) e = nc.memset32(bp->counters, 0u, gs.size() + 1);
  for (size_t gi = 0; e == cudaSuccess && gi < launches.size(); ++gi)
    e = stencil_node(launches[gi], grids[gi], blocks[gi], smems[gi], nc);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&bp->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_fail(e, "building the batched launch graph");
  return MRW_OK;
}

}  // namespace

extern "C" {

mrw_status mrw_execute_batched(mrw_node_t root, const uint8_t *in_arena, uint8_t *out_arena, int64_t arena_bytes,
                               const int64_t *desc, int64_t n, const mrw_config *cfg, void *stream,
                               mrw_future_t *out) {
  if (!out) return fail(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!in_arena || !out_arena || !desc || n <= 0 || arena_bytes <= 0)
    return fail(MRW_ERR_INVALID_ARG, "batched call needs arenas, descriptors and n > 0");
  if (n > (1 << 24)) return fail(MRW_ERR_INVALID_ARG, "too many instances");
  if ((uintptr_t)in_arena % 16 || (uintptr_t)out_arena % 16)
    return fail(MRW_ERR_CONSTRAINT, "arenas must be 16-byte aligned");
  {
    const uintptr_t a0 = (uintptr_t)in_arena, b0 = (uintptr_t)out_arena;
    if (a0 < b0 + arena_bytes && b0 < a0 + arena_bytes) return fail(MRW_ERR_INVALID_ARG, "arenas overlap");
  }
  Program p;
  TRY(get_program(root, &p));
  if (p.fam != F_IMAGE) return fail(MRW_ERR_UNSUPPORTED, "batched execution runs image trees");
  if (p.reduce != RED_NONE) return fail(MRW_ERR_UNSUPPORTED, "batched MapReduce");
  if (p.while_begin >= 0) return fail(MRW_ERR_UNSUPPORTED, "batched WHILE_CHANGED loops");
  for (const ImgStage &st : p.img)
    if (st.kind == OP_USER) return fail(MRW_ERR_UNSUPPORTED, "user-defined stages in a batched call");
  for (int64_t i = 0; i < n; ++i) {
    const int64_t off = desc[5 * i], W = desc[5 * i + 1], H = desc[5 * i + 2], pitch = desc[5 * i + 3];
    if (W < 1 || H < 1 || W > (1 << 20) || H > (1 << 20)) return fail(MRW_ERR_SHAPE, "instance %lld: bad size", (long long)i);
    if (off < 0 || off % 16 || pitch % 16 || pitch < W || pitch > INT32_MAX)
      return fail(MRW_ERR_CONSTRAINT, "instance %lld: offset and pitch must be multiples of 16, pitch >= W",
                  (long long)i);
    if (off > arena_bytes || H * pitch > arena_bytes - off)  // H * pitch < 2^51: no overflow
      return fail(MRW_ERR_SHAPE, "instance %lld lies outside the arena", (long long)i);
  }
  mrw_config c = cfg ? *cfg : default_config(F_IMAGE);
  TRY(check_config(c));
  Launch L;
  TRY(begin_launch(L, stream));
  char keyb[256];
  const uint64_t dh = hash_bytes(desc, (size_t)n * 5 * sizeof(int64_t));
  snprintf(keyb, sizeof keyb, "%d|%p|%p|%p|%lld|%llx|%lld|%d,%d,%d,%d,%d,%d", L.device, (void *)stream,
           (const void *)in_arena, (void *)out_arena, (long long)arena_bytes, (unsigned long long)dh, (long long)n,
           c.fusion, c.block, c.ctas_per_sm, c.tile_rows, c.tile_cols, c.unroll);
  const std::string key = tree_signature(root) + "|" + keyb;
  std::shared_ptr<BatchPlan> cached = batch_plans().find(key);
  if (!cached) {
    BatchPlan built;
    mrw_status s = build_batch_plan(L, p, in_arena, out_arena, arena_bytes, desc, n, c, &built);
    if (s != MRW_OK) {
      destroy_batch_plan(built);
      return s;
    }
    TRY(make_cached(built, destroy_batch_plan, &cached));
    cached = batch_plans().insert(key, cached);
  }
  const BatchPlan &plan = *cached;
  mrw_future *f = new (std::nothrow) mrw_future();
  if (!f) return fail(MRW_ERR_OOM, "future");
  f->device = L.device;
  mrw_status s = status_pool().take(&f->slot);
  if (s == MRW_OK) s = take_future_events(f, false);
  if (s != MRW_OK) {
    free_future(f);
    return s;
  }
  cudaError_t e = cudaGraphLaunch(plan.exec, L.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f->slot.host, plan.counters + plan.ngroups, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                        L.stream);
  cudaEventRecord(plan.last_use, L.stream);
  f->has_status = true;
  cudaEventRecord(f->done, L.stream);
  if (e != cudaSuccess) {
    cudaEventSynchronize(f->done);
    free_future(f);
    return cuda_fail(e, "launching the batched graph");
  }
  *out = f;
  return MRW_OK;
}

}  // extern "C"

// ============================================================================================
// Plan description, features, tuner, knowledge base, cost model
// ============================================================================================
namespace {

const char *op_name(int k) {
  switch (k) {
    case OP_NOISE: return "noise";
    case OP_SOLARISE: return "solarise";
    case OP_MIRROR: return "mirror";
    case OP_BLUR: return "blur5";
    case OP_THRESH: return "threshold3";
    case OP_USER: return "user";
  }
  return "?";
}

const char *pattern_name(int32_t pat) {
  switch (pat) {
    case PAT_NONE: return "none";
    case PAT_NOISE: return "noise";
    case PAT_SOLARISE: return "solarise";
    case PAT_NOISE_SOLARISE: return "noise_solarise";
    case PAT_THRESH: return "threshold3";
  }
  return "generic";
}

void ops_json(std::ostringstream &o, const std::vector<ImgStage> &v) {
  o << "[";
  for (size_t i = 0; i < v.size(); ++i)
    o << (i ? "," : "") << "\"" << (v[i].kind == OP_USER ? "user:" + v[i].fn->name : std::string(op_name(v[i].kind)))
      << "\"";
  o << "]";
}

mrw_status describe(const Program &p, const mrw_buffer *args, int nargs, const mrw_config &c, int sms,
                    std::string *out) {
  std::ostringstream o;
  if (p.fam == F_IMAGE) {
    View vin, vout, vred;
    TRY(validate_image_args(p, args, nargs, &vin, &vout, &vred));
    const ImgGeom geo = geom_of(args[0], vin);
    const std::vector<Group> gs = group_stages(p, c.fusion == MRW_FUSE_ALL, false);
    const bool chunked = p.while_begin < 0 && chunked_staging(gs, vin, vout, geo);
    o << "{\"family\":\"image\",\"W\":" << geo.W << ",\"H\":" << geo.H << ",\"D\":" << geo.D
      << ",\"reduce\":" << p.reduce << ",\"staging\":\"" << (chunked ? "chunked" : "whole") << "\"";
    if (p.while_begin >= 0)
      o << ",\"while_changed\":{\"first_stage\":" << p.while_begin << ",\"end_stage\":" << p.while_end
        << ",\"max_iters\":" << p.while_max << ",\"body_kernels\":"
        << group_stages(sub_program(p, p.while_begin, p.while_end), c.fusion == MRW_FUSE_ALL, false).size() << "}";
    o << ",\"groups\":[";
    for (size_t i = 0; i < gs.size(); ++i) {
      const Group &g = gs[i];
      o << (i ? "," : "") << "{";
      if (g.user) {
        o << "\"kernel\":\"user_chain\",\"ops\":";
        ops_json(o, g.pre);
      } else if (g.use_stencil) {
        StencilArgs sa{};
        fill_stencil_ops(g, sa);
        const StencilShape s = stencil_shape(c, sa);
        const int64_t tx = (geo.W + s.tile_w - 1) / s.tile_w, ty = (geo.H + s.tile_h - 1) / s.tile_h;
        o << "\"kernel\":\"" << (sa.rows_kernel ? "stencil_rows" : "stencil") << "\",\"pre\":";
        ops_json(o, g.pre);
        uint32_t pt = 0;
        o << ",\"pre_pattern\":\"" << pattern_name(op_pattern(sa.pre, sa.npre, &pt)) << "\"";
        o << ",\"blur\":" << (g.blur ? "true" : "false") << ",\"suf\":";
        ops_json(o, g.suf);
        o << ",\"tile\":[" << s.tile_h << "," << s.tile_w << "],\"box\":[" << s.box_h << "," << s.box_w
          << "],\"tiles_x\":" << tx << ",\"tiles_y\":" << ty << ",\"tiles\":" << tx * ty * geo.D
          << ",\"grid\":" << stencil_grid(s, sa, tx * ty * geo.D, sms) << ",\"block\":" << s.block
          << ",\"smem\":" << s.smem;
      } else {
        const ChainShape s = chain_shape(c, sms, geo.W, geo.rows, p.wg, count_noise(g.pre), false, false);
        o << "\"kernel\":\"chain\",\"ops\":";
        ops_json(o, g.pre);
        ChainOp ops[kMaxChainOps];
        fill_ops(g.pre, mirror_parity(g.pre), ops);
        uint32_t pt = 0;
        o << ",\"pattern\":\"" << pattern_name(op_pattern(ops, (int)g.pre.size(), &pt)) << "\"";
        o << ",\"reduce_only\":" << (g.reduce_only ? "true" : "false") << ",\"reduce\":" << g.reduce
          << ",\"nu\":16,\"col_vecs\":" << (geo.W + 15) / 16 << ",\"rows_parallel\":" << s.rows_parallel
          << ",\"grid\":" << s.grid << ",\"block\":" << s.block << ",\"unroll\":" << s.unroll
          << ",\"order\":\"" << (s.blocked ? "blocked" : "persistent") << "\""
          << ",\"finish_kernel\":" << (g.reduce != RED_NONE && !chunked ? "true" : "false");
      }
      o << "}";
    }
    o << "]}";
  } else if (p.fam == F_NBODY) {
    if (nargs != 3) return fail(MRW_ERR_INVALID_ARG, "N-body trees take x, v, a");
    const int64_t n = args[0].shape[0];
    const NbShape s = nbody_shape(c, sms, n, p.wg);
    o << "{\"family\":\"nbody\",\"n\":" << n << ",\"grid\":" << s.grid << ",\"block\":" << s.block
      << ",\"j_groups\":4,\"threads_per_group\":" << s.block / 4 << ",\"bodies_per_thread\":" << s.bpt
      << ",\"steps\":[";
    for (size_t i = 0; i < p.nb.size(); ++i) {
      const NbStep &st = p.nb[i];
      o << (i ? "," : "") << "{\"kind\":\"" << (st.accel ? "accel" : "kdk") << "\",\"iters\":" << st.iters
        << ",\"loop\":\""
        << (st.accel ? "none" : (c.fusion == MRW_FUSE_NONE ? "host" : (st.from_loop ? "device_graph" : "unrolled")))
        << "\"}";
    }
    o << "],\"partitions\":[";
    for (int cta = 0; cta < s.grid; ++cta) {
      const int64_t lo = n * cta / s.grid, hi = n * (cta + 1) / s.grid;
      o << (cta ? "," : "") << "[" << lo << "," << hi - lo << "]";
    }
    o << "]}";
  } else if (p.fam == F_FFT) {
    View vx, vy;
    TRY(validate_fft_args(args, nargs, &vx, &vy));
    const int per = c.fusion == MRW_FUSE_ALL ? kFftMaxSteps : 1;
    const FftForm form = fft_form(c, vx.rows);
    const bool c16 = form == FFT_C16, tm = form == FFT_TMEM, l2 = form == FFT_L2;
    o << "{\"family\":\"fft\",\"n\":" << kFftN << ",\"nfft\":" << vx.rows << ",\"form\":\""
      << (l2 ? "l2" : (c16 ? "c16" : (tm ? "tmem" : "reg"))) << "\"";
    if (l2) {
      FftL2Plan pl{};
      const int ctas = fft_l2_ctas_per_sm() * sms;
      if (!fft_l2_plan(vx.rows, (int)std::min<size_t>(per, p.fft.size()), ctas, &pl))
        return fail(MRW_ERR_UNSUPPORTED, "%lld FFT rows do not fit the L2-ring schedule", (long long)vx.rows);
      o << ",\"cluster\":1,\"smem\":" << fft_l2_smem_bytes() << ",\"tmem\":false,\"ctas\":" << pl.ctas
        << ",\"ctas_per_sm\":" << fft_l2_ctas_per_sm() << ",\"slice_rows\":" << pl.sc.G << ",\"lag_steps\":" << pl.sc.L
        << ",\"ring_rows\":" << pl.ring_rows << ",\"schedule_ok\":"
        << (fft_l2_schedule_ok(pl.sc, pl.ring_rows) ? "true" : "false");
    } else {
      o << ",\"cluster\":" << (c16 ? kFft16Cluster : kFftCluster) << ",\"smem\":"
        << (c16 ? fft16_smem_bytes() : fft_smem_bytes()) << ",\"tmem\":" << (tm ? "true" : "false")
        << ",\"clusters_resident\":" << (c16 ? fft16_max_clusters() : fft_max_clusters(tm));
    }
    o << ",\"launches\":[";
    for (size_t i = 0; i < p.fft.size(); i += per) {
      o << (i ? "," : "") << "[";
      for (size_t k = i; k < std::min(p.fft.size(), i + per); ++k) o << (k > i ? "," : "") << (p.fft[k] > 0 ? "\"fft\"" : "\"ifft\"");
      o << "]";
    }
    o << "]}";
  } else {
    View vx, vy;
    TRY(validate_saxpy_args(args, nargs, &vx, &vy));
    const size_t per = c.fusion == MRW_FUSE_ALL ? (size_t)kMaxSaxpyStages : 1;
    const int unroll = c.unroll ? c.unroll : 4;
    o << "{\"family\":\"saxpy\",\"n\":" << vx.numel() << ",\"stages\":" << p.alphas.size()
      << ",\"launches\":" << (p.alphas.size() + per - 1) / per << ",\"unroll\":" << unroll
      << ",\"block\":256,\"grid\":" << saxpy_grid(vx.numel(), unroll) << "}";
  }
  *out = o.str();
  return MRW_OK;
}

float flog2(double v) { return v > 0 ? (float)std::log2(v) : 0.f; }

mrw_status features_of(const Program &p, const mrw_buffer *args, int nargs, float *f) {
  for (int i = 0; i < MRW_NFEATURES; ++i) f[i] = 0.f;
  if (nargs < 1 || !args) return fail(MRW_ERR_INVALID_ARG, "features need the arguments");
  View v;
  TRY(view_of(args[0], 0, &v));
  f[0] = p.fam == F_IMAGE;
  f[1] = p.fam == F_SAXPY;
  f[2] = p.fam == F_NBODY;
  f[3] = p.reduce != RED_NONE;
  int nn = 0, npw = 0, nm = 0, nb = 0;
  for (const ImgStage &s : p.img) {
    nn += s.kind == OP_NOISE;
    npw += s.kind == OP_SOLARISE || s.kind == OP_THRESH || s.kind == OP_USER;
    nm += s.kind == OP_MIRROR;
    nb += s.kind == OP_BLUR;
  }
  const double stages = p.fam == F_IMAGE ? (double)p.img.size()
                        : (p.fam == F_SAXPY ? (double)p.alphas.size() : (p.fam == F_FFT ? (double)p.fft.size() : 0.0));
  f[4] = (float)stages;
  f[5] = (float)nn;
  f[6] = (float)npw;
  f[7] = (float)nm;
  f[8] = (float)nb;
  const double numel = (double)v.numel();
  f[9] = flog2(numel);
  f[10] = flog2((double)v.width);
  f[11] = flog2((double)v.rows);
  f[12] = (v.width * v.esize) % 16 != 0;
  f[13] = (float)v.esize;
  double bytes = 0, ops = 0;
  if (p.fam == F_IMAGE) {
    bytes = 2.0 * numel + (p.reduce ? 8.0 : 0.0);
    ops = 20.0 * nn + 2.0 * npw + 15.0 * nb + 0.5 * nm;
  } else if (p.fam == F_SAXPY) {
    bytes = 12.0 * numel;
    ops = 2.0 * stages;
  } else if (p.fam == F_FFT) {
    bytes = 16.0 * numel;
    ops = 5.0 * 16.0 * stages;  // 5 N log2 N flops per transform, per value
  } else {
    bytes = 48.0 * numel;
    ops = 20.0 * numel;
  }
  f[14] = flog2(bytes);
  f[15] = (float)(ops / 16.0);
  return MRW_OK;
}

std::vector<mrw_config> candidates_for(Family fam) {
  std::vector<mrw_config> v;
  for (int i = 0; i < 16; ++i) v.push_back(fam == F_NBODY ? nbody_candidate(i) : candidate(i));
  return v;
}

// Median device time of `reps` executions of one configuration (after one warm-up).
mrw_status time_config(const Program &p, const mrw_buffer *args, int nargs, const mrw_config &c, int reps,
                       void *stream, unsigned int *status, float *ms) {
  Launch L;
  TRY(begin_launch(L, stream));
  bool used = false;
  mrw_status s = enqueue(L, p, args, nargs, c, status, &used);
  L.free_all();
  if (s != MRW_OK) return s;
  std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
  for (auto &e : ev) CU(cudaEventCreate(&e));
  for (int r = 0; r < reps && s == MRW_OK; ++r) {
    cudaEventRecord(ev[2 * r], L.stream);
    s = enqueue(L, p, args, nargs, c, status, &used);
    L.free_all();
    cudaEventRecord(ev[2 * r + 1], L.stream);
  }
  const cudaError_t e = cudaStreamSynchronize(L.stream);
  std::vector<float> t;
  for (int r = 0; r < reps && s == MRW_OK && e == cudaSuccess; ++r) {
    float x = 0;
    cudaEventElapsedTime(&x, ev[2 * r], ev[2 * r + 1]);
    t.push_back(x);
  }
  for (auto &ee : ev) cudaEventDestroy(ee);
  if (e != cudaSuccess) return cuda_fail(e, "timing run");
  if (s != MRW_OK) return s;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return MRW_OK;
}

}  // namespace

// --------------------------------------------------------------------------------------------
// Model helpers (host side)
// --------------------------------------------------------------------------------------------
namespace {

mrw_status model_predict(mrw_model *m, const float *feat, int *best) {
  int cur;
  CU(cudaGetDevice(&cur));
  if (cur != m->device) CU(cudaSetDevice(m->device));
  float *buf = nullptr;
  mrw_status s = MRW_OK;
  cudaError_t e = cudaMalloc(&buf, sizeof(float) * (MRW_NFEATURES + m->d.k));
  if (e == cudaSuccess) e = cudaMemcpy(buf, feat, sizeof(float) * MRW_NFEATURES, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_mlp_forward(m->d, m->bf, buf, 1, buf + MRW_NFEATURES, nullptr);
  std::vector<float> y((size_t)m->d.k);
  if (e == cudaSuccess)
    e = cudaMemcpy(y.data(), buf + MRW_NFEATURES, sizeof(float) * m->d.k, cudaMemcpyDeviceToHost);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) s = cuda_fail(e, "cost-model inference");
  if (cur != m->device) cudaSetDevice(cur);
  if (s != MRW_OK) return s;
  *best = (int)(std::min_element(y.begin(), y.end()) - y.begin());
  return MRW_OK;
}

}  // namespace

extern "C" {

mrw_status mrw_fft_schedule_check(int64_t nfft, int32_t nsteps, int32_t ctas, int64_t *out) {
  FftL2Plan pl{};
  if (!fft_l2_plan(nfft, nsteps, ctas, &pl))
    return fail(MRW_ERR_UNSUPPORTED, "no L2-ring schedule for %lld rows, %d transforms, %d CTAs", (long long)nfft,
                nsteps, ctas);
  if (out) {
    out[0] = pl.sc.G;
    out[1] = pl.sc.L;
    out[2] = pl.ring_rows;
    out[3] = pl.ctas;
    out[4] = fsch_total_tickets(pl.sc);
  }
  if (!fft_l2_schedule_ok(pl.sc, pl.ring_rows))
    return fail(MRW_ERR_CONSTRAINT, "the L2-ring schedule for %lld rows is inconsistent", (long long)nfft);
  return MRW_OK;
}

mrw_status mrw_plan_describe(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfg,
                             char *buf, int64_t cap, int64_t *needed) {
  Program p;
  TRY(get_program(root, &p));
  if (nargs < 0 || (nargs && !args)) return fail(MRW_ERR_INVALID_ARG, "bad argument list");
  const mrw_config c = cfg ? *cfg : pick_config(root, p, args, nargs);
  TRY(check_config(c));
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) sms = v;
  } else {
    cudaGetLastError();
  }
  std::string s;
  TRY(describe(p, args, nargs, c, sms, &s));
  if (needed) *needed = (int64_t)s.size() + 1;
  if (buf && cap > 0) {
    const size_t n = std::min<size_t>((size_t)cap - 1, s.size());
    memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return MRW_OK;
}

mrw_status mrw_features(mrw_node_t root, const mrw_buffer *args, int32_t nargs, float *feat16) {
  if (!feat16) return fail(MRW_ERR_INVALID_ARG, "feat16 is NULL");
  Program p;
  TRY(get_program(root, &p));
  return features_of(p, args, nargs, feat16);
}

mrw_status mrw_tune_candidates(mrw_node_t root, const mrw_buffer *args, int32_t nargs, mrw_config *cfgs, int32_t cap,
                               int32_t *count) {
  (void)args;
  (void)nargs;
  if (!count) return fail(MRW_ERR_INVALID_ARG, "count is NULL");
  Program p;
  TRY(get_program(root, &p));
  const std::vector<mrw_config> v = candidates_for(p.fam);
  *count = (int32_t)v.size();
  if (cfgs)
    for (int i = 0; i < cap && i < (int)v.size(); ++i) cfgs[i] = v[i];
  return MRW_OK;
}

mrw_status mrw_tune_measure(mrw_node_t root, const mrw_buffer *args, int32_t nargs, const mrw_config *cfgs,
                            int32_t ncfg, int32_t reps, void *stream, float *times_ms) {
  if (!cfgs || !times_ms || ncfg < 0 || reps < 1 || reps > 1000) return fail(MRW_ERR_INVALID_ARG, "bad arguments");
  Program p;
  TRY(get_program(root, &p));
  for (int i = 0; i < nargs; ++i)
    if (args[i].memory != MRW_MEM_DEVICE) return fail(MRW_ERR_INVALID_ARG, "the tuner times device buffers");
  StatusSlot slot;
  TRY(status_pool().take(&slot));
  for (int i = 0; i < ncfg; ++i) {
    float ms = -1.f;
    const mrw_status s = time_config(p, args, nargs, cfgs[i], reps, stream, slot.dev, &ms);
    if (s == MRW_ERR_CUDA || s == MRW_ERR_OOM) {
      status_pool().give(slot);
      return s;
    }
    times_ms[i] = s == MRW_OK ? ms : -1.f;
  }
  status_pool().give(slot);
  return MRW_OK;
}

mrw_status mrw_tune(mrw_node_t root, const mrw_buffer *args, int32_t nargs, mrw_tune_mode mode, int32_t reps,
                    void *stream, mrw_config *best, float *best_ms) {
  Program p;
  TRY(get_program(root, &p));
  const std::vector<mrw_config> cands = candidates_for(p.fam);
  mrw_config pick = default_config(p.fam);
  float pick_ms = -1.f;
  if (mode == MRW_TUNE_EXHAUSTIVE) {
    std::vector<float> t(cands.size());
    TRY(mrw_tune_measure(root, args, nargs, cands.data(), (int32_t)cands.size(), reps, stream, t.data()));
    for (size_t i = 0; i < t.size(); ++i)
      if (t[i] >= 0 && (pick_ms < 0 || t[i] < pick_ms)) {
        pick_ms = t[i];
        pick = cands[i];
      }
  } else if (mode == MRW_TUNE_PRUNED) {
    // Algorithm 1's ordered search: fusion modes in order (fused first), then launch shapes in order
    // of expected benefit; a dimension stops at the first candidate that does not improve the best.
    for (int f = 0; f < 2; ++f) {
      float best_f = -1.f;
      for (int sidx = 0; sidx < 8; ++sidx) {
        const mrw_config &c = cands[(size_t)(8 * f + sidx)];
        float ms = -1.f;
        TRY(mrw_tune_measure(root, args, nargs, &c, 1, reps, stream, &ms));
        if (ms < 0) continue;
        const bool improved = best_f < 0 || ms < best_f;
        if (improved) best_f = ms;
        if (pick_ms < 0 || ms < pick_ms) {
          pick_ms = ms;
          pick = c;
        }
        if (!improved) break;  // discard the remaining shapes of this fusion mode
      }
      if (f == 0 && best_f >= 0 && pick_ms < best_f) break;
      if (f == 1 && best_f > pick_ms) break;
    }
  } else if (mode == MRW_TUNE_MODEL) {
    mrw_model *m = nullptr;
    std::vector<mrw_config> cfgs;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      m = installed_model().model;
      cfgs = installed_model().cfgs;
    }
    if (!m || (int)cfgs.size() != m->d.k) return fail(MRW_ERR_INVALID_ARG, "no cost model installed");
    float f[MRW_NFEATURES];
    TRY(features_of(p, args, nargs, f));
    int b = 0;
    TRY(model_predict(m, f, &b));
    pick = cfgs[(size_t)b];
  } else {
    return fail(MRW_ERR_INVALID_ARG, "unknown tune mode");
  }
  const std::string key = tree_signature(root) + "|" + workload_signature(args, nargs);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    kb()[key] = {pick, pick_ms, (int)mode};
    bump_plan_gen();
  }
  if (best) *best = pick;
  if (best_ms) *best_ms = pick_ms;
  return MRW_OK;
}

mrw_status mrw_kb_save(const char *path) {
  if (!path) return fail(MRW_ERR_INVALID_ARG, "path is NULL");
  std::ofstream f(path);
  if (!f) return fail(MRW_ERR_INVALID_ARG, "cannot write %s", path);
  std::lock_guard<std::mutex> lk(g_mu);
  for (const auto &kv : kb()) {
    const mrw_config &c = kv.second.cfg;
    f << kv.first << "\t" << c.fusion << " " << c.block << " " << c.ctas_per_sm << " " << c.tile_rows << " "
      << c.tile_cols << " " << c.unroll << "\t" << kv.second.ms << "\t" << kv.second.source << "\n";
  }
  return f ? MRW_OK : fail(MRW_ERR_INVALID_ARG, "write failed: %s", path);
}

mrw_status mrw_kb_load(const char *path) {
  if (!path) return fail(MRW_ERR_INVALID_ARG, "path is NULL");
  std::ifstream f(path);
  if (!f) return fail(MRW_ERR_INVALID_ARG, "cannot read %s", path);
  std::string line;
  std::map<std::string, KbRecord> add;
  while (std::getline(f, line)) {
    while (!line.empty() && (line.back() == '\r' || line.back() == ' ')) line.pop_back();
    if (line.empty()) continue;
    const size_t t1 = line.find('\t'), t2 = line.find('\t', t1 + 1), t3 = line.find('\t', t2 + 1);
    if (t1 == std::string::npos || t2 == std::string::npos || t3 == std::string::npos)
      return fail(MRW_ERR_INVALID_ARG, "malformed knowledge-base line");
    KbRecord r{};
    std::istringstream cs(line.substr(t1 + 1, t2 - t1 - 1));
    cs >> r.cfg.fusion >> r.cfg.block >> r.cfg.ctas_per_sm >> r.cfg.tile_rows >> r.cfg.tile_cols >> r.cfg.unroll;
    if (!cs || check_config(r.cfg) != MRW_OK) return fail(MRW_ERR_INVALID_ARG, "malformed configuration in %s", path);
    // strtof / strtol rather than the throwing std::sto*: nothing may throw across the C ABI
    const std::string ms = line.substr(t2 + 1, t3 - t2 - 1), src = line.substr(t3 + 1);
    char *e1 = nullptr, *e2 = nullptr;
    r.ms = strtof(ms.c_str(), &e1);
    const long so = strtol(src.c_str(), &e2, 10);
    if (ms.empty() || src.empty() || *e1 != '\0' || *e2 != '\0' || so < INT32_MIN || so > INT32_MAX)
      return fail(MRW_ERR_INVALID_ARG, "malformed time or source field in %s", path);
    r.source = (int)so;
    add[line.substr(0, t1)] = r;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &kv : add) kb()[kv.first] = kv.second;
  bump_plan_gen();
  return MRW_OK;
}

mrw_status mrw_kb_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  kb().clear();
  bump_plan_gen();
  return MRW_OK;
}

int64_t mrw_kb_size(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  return (int64_t)kb().size();
}

// --------------------------------------------------------------------------------------------
// Cost model
// --------------------------------------------------------------------------------------------
mrw_status mrw_model_create(int32_t k, int32_t hidden, uint64_t seed, mrw_model_t *out) {
  if (!out) return fail(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > 64 || hidden < 1 || hidden > 128) return fail(MRW_ERR_INVALID_ARG, "K in 1..64, hidden in 1..128");
  mrw_model *m = new (std::nothrow) mrw_model();
  if (!m) return fail(MRW_ERR_OOM, "model");
  m->d = mlp_dims(MRW_NFEATURES, hidden, k);
  const int64_t np = m->d.nparams;
  cudaGetDevice(&m->device);
  cudaError_t e = cudaMalloc(&m->master, sizeof(float) * (size_t)(4 * np + 1));
  if (e == cudaSuccess) e = cudaMalloc(&m->bf, sizeof(uint16_t) * (size_t)np);
  if (e != cudaSuccess) {
    mrw_model_release(m);
    return cuda_fail(e, "model buffers");
  }
  m->m = m->master + np;
  m->v = m->m + np;
  m->grads = m->v + np;
  m->loss = m->grads + np;
  // He-uniform weights, zero biases
  std::mt19937_64 rng(seed);
  std::vector<float> h((size_t)np, 0.f);
  auto he = [&](int64_t off, int64_t fan_out, int64_t fan_in) {
    std::uniform_real_distribution<float> u(-std::sqrt(6.f / fan_in), std::sqrt(6.f / fan_in));
    for (int64_t i = 0; i < fan_out * fan_in; ++i) h[(size_t)(off + i)] = u(rng);
  };
  he(m->d.off_w1, hidden, MRW_NFEATURES);
  he(m->d.off_w2, hidden, hidden);
  he(m->d.off_w3, k, hidden);
  const mrw_status s = mrw_model_set_params(m, h.data());
  if (s != MRW_OK) {
    mrw_model_release(m);
    return s;
  }
  *out = m;
  return MRW_OK;
}

void mrw_model_release(mrw_model_t m) {
  if (!m) return;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (installed_model().model == m) {
      installed_model().model = nullptr;
      installed_model().cfgs.clear();
    }
  }
  if (m->master) cudaFree(m->master);
  if (m->bf) cudaFree(m->bf);
  if (m->idx) cudaFree(m->idx);
  delete m;
}

int64_t mrw_model_num_params(mrw_model_t m) { return m ? m->d.nparams : 0; }

mrw_status mrw_model_set_params(mrw_model_t m, const float *host_params) {
  if (!m || !host_params) return fail(MRW_ERR_INVALID_ARG, "NULL argument");
  const int64_t np = m->d.nparams;
  CU(cudaMemcpy(m->master, host_params, sizeof(float) * (size_t)np, cudaMemcpyHostToDevice));
  CU(cudaMemset(m->m, 0, sizeof(float) * (size_t)(3 * np + 1)));
  CU(launch_mlp_round_bf16(m->master, m->bf, np, nullptr));
  CU(cudaDeviceSynchronize());
  m->step = 0;
  return MRW_OK;
}

mrw_status mrw_model_get_params(mrw_model_t m, float *host_params) {
  if (!m || !host_params) return fail(MRW_ERR_INVALID_ARG, "NULL argument");
  CU(cudaMemcpy(host_params, m->master, sizeof(float) * (size_t)m->d.nparams, cudaMemcpyDeviceToHost));
  return MRW_OK;
}

mrw_status mrw_model_forward(mrw_model_t m, const float *x, int64_t n, float *y, void *stream) {
  if (!m || (n > 0 && (!x || !y)) || n < 0) return fail(MRW_ERR_INVALID_ARG, "bad arguments");
  CU(launch_mlp_forward(m->d, m->bf, x, n, y, (cudaStream_t)stream));
  return MRW_OK;
}

mrw_status mrw_model_gradients(mrw_model_t m, const float *x, const float *t, int64_t n, float *grads, float *loss,
                               void *stream) {
  if (!m || !x || !t || !grads || n < 1) return fail(MRW_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaMemsetAsync(grads, 0, sizeof(float) * (size_t)m->d.nparams, s));
  CU(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
  CU(launch_mlp_backward(m->d, m->bf, x, t, nullptr, n, 1.f / (float)(n * m->d.k), grads, m->loss, s));
  float l = 0;
  CU(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (loss) *loss = l / (float)(n * m->d.k);
  return MRW_OK;
}

mrw_status mrw_model_adam_step(mrw_model_t m, const float *grads, float lr, void *stream) {
  if (!m || !grads) return fail(MRW_ERR_INVALID_ARG, "bad arguments");
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->step));
  const float bc2 = (float)(1.0 - std::pow(0.999, (double)m->step));
  CU(launch_mlp_adam(m->master, m->m, m->v, grads, m->d.nparams, lr, b1, b2, 1e-8f, bc1, bc2, m->bf,
                     (cudaStream_t)stream));
  return MRW_OK;
}

mrw_status mrw_model_train(mrw_model_t m, const float *x, const float *t, int64_t n, int32_t epochs, int32_t batch,
                           float lr, uint64_t seed, void *stream, float *final_loss) {
  if (!m || !x || !t || n < 1 || epochs < 0 || batch < 1) return fail(MRW_ERR_INVALID_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (m->idx_cap < n) {
    if (m->idx) cudaFree(m->idx);
    m->idx = nullptr;
    m->idx_cap = 0;
    CU(cudaMalloc(&m->idx, sizeof(int32_t) * (size_t)n));
    m->idx_cap = n;
  }
  std::vector<int32_t> order((size_t)n);
  for (int64_t i = 0; i < n; ++i) order[(size_t)i] = (int32_t)i;
  std::mt19937_64 rng(seed);
  float last = 0.f;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    CU(cudaMemcpyAsync(m->idx, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int64_t cnt = std::min<int64_t>(batch, n - b0);
      CU(cudaMemsetAsync(m->grads, 0, sizeof(float) * (size_t)m->d.nparams, s));
      CU(launch_mlp_backward(m->d, m->bf, x, t, m->idx + b0, cnt, 1.f / (float)(cnt * m->d.k), m->grads, m->loss, s));
      TRY(mrw_model_adam_step(m, m->grads, lr, s));
    }
    float l = 0;
    CU(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));  // `order` is reshuffled next epoch
    last = l / (float)(n * m->d.k);
  }
  if (final_loss) *final_loss = last;
  return MRW_OK;
}

mrw_status mrw_tune_set_model(mrw_model_t m, const mrw_config *cfgs, int32_t k) {
  std::lock_guard<std::mutex> lk(g_mu);
  bump_plan_gen();
  if (!m) {
    installed_model().model = nullptr;
    installed_model().cfgs.clear();
    return MRW_OK;
  }
  if (!cfgs || k != m->d.k) return fail(MRW_ERR_INVALID_ARG, "the model needs one configuration per output");
  for (int i = 0; i < k; ++i) TRY(check_config(cfgs[i]));
  installed_model().model = m;
  installed_model().cfgs.assign(cfgs, cfgs + k);
  return MRW_OK;
}

}  // extern "C"

// ============================================================================================
// Allocation-free batched execution
// ============================================================================================
namespace {

// Image stages of a tree, depth first, into a fixed array (no heap allocation).
mrw_status collect_image_stages(const mrw_node *n, ImgStage *out, int *cnt, int cap, int depth) {
  if (depth > 64) return fail(MRW_ERR_UNSUPPORTED, "tree deeper than 64 levels");
  switch (n->kind) {
    case N_STAGE: {
      if (n->user) return fail(MRW_ERR_UNSUPPORTED, "user-defined stages in the allocation-free batched call");
      const int ok = op_kind_of(n->stage);
      if (ok < 0) return fail(MRW_ERR_UNSUPPORTED, "the allocation-free batched call runs image stages only");
      if (*cnt >= cap) return fail(MRW_ERR_UNSUPPORTED, "more than %d image stages", cap);
      const mrw_stage_params &q = n->params;
      if (n->stage == MRW_ST_THRESHOLD3 && (q.t0 < 0 || q.t0 > 255 || q.t1 < 0 || q.t1 > 255))
        return fail(MRW_ERR_INVALID_ARG, "threshold outside [0, 255]");
      out[(*cnt)++] = {ok, q.seed, (uint32_t)(q.t0 & 0xFF) | ((uint32_t)(q.t1 & 0xFF) << 8), q.nu, q.wg};
      return MRW_OK;
    }
    case N_PIPELINE:
      if (n->kids.empty()) return fail(MRW_ERR_INVALID_ARG, "empty pipeline");
      for (const mrw_node *c : n->kids) TRY(collect_image_stages(c, out, cnt, cap, depth + 1));
      return MRW_OK;
    case N_MAP:
      return collect_image_stages(n->kids[0], out, cnt, cap, depth + 1);
    case N_LOOP:
      if (n->loop.kind != MRW_LOOP_FOR) return fail(MRW_ERR_UNSUPPORTED, "loop kind %d", n->loop.kind);
      for (int64_t i = 0; i < n->loop.max_iters; ++i) TRY(collect_image_stages(n->kids[0], out, cnt, cap, depth + 1));
      return MRW_OK;
    case N_MAPREDUCE:
      return fail(MRW_ERR_UNSUPPORTED, "batched MapReduce");
  }
  return fail(MRW_ERR_INVALID_ARG, "bad node");
}

void fill_ops_array(const ImgStage *v, int n, ChainOp *ops, int *parity) {
  int m = 0;
  for (int i = 0; i < n; ++i) m ^= (v[i].kind == OP_MIRROR);
  int before = 0;
  for (int i = 0; i < n; ++i) {
    ops[i].kind = v[i].kind;
    ops[i].seed = v[i].seed;
    ops[i].t = v[i].t;
    ops[i].flip = m ^ (before & 1);
    before += v[i].kind == OP_MIRROR;
  }
  *parity = m;
}

}  // namespace

extern "C" mrw_status mrw_execute_batched_noalloc(mrw_node_t root, const uint8_t *in_arena, uint8_t *out_arena,
                                                  int64_t arena_bytes, const int64_t *desc, int64_t n,
                                                  const mrw_config *cfg, void *stream) {
  if (!root || !in_arena || !out_arena || !desc || arena_bytes <= 0)
    return fail(MRW_ERR_INVALID_ARG, "the allocation-free batched call needs a tree, arenas and descriptors");
  if (n < 1 || n > MRW_NOALLOC_MAX_INSTANCES)
    return fail(MRW_ERR_INVALID_ARG, "the allocation-free batched call takes 1 to %d instances, got %lld",
                MRW_NOALLOC_MAX_INSTANCES, (long long)n);
  if ((uintptr_t)in_arena % 16 || (uintptr_t)out_arena % 16)
    return fail(MRW_ERR_CONSTRAINT, "arenas must be 16-byte aligned");
  {
    const uintptr_t a0 = (uintptr_t)in_arena, b0 = (uintptr_t)out_arena;
    if (a0 < b0 + arena_bytes && b0 < a0 + arena_bytes) return fail(MRW_ERR_INVALID_ARG, "arenas overlap");
  }
  for (int64_t i = 0; i < n; ++i) {
    const int64_t off = desc[5 * i], W = desc[5 * i + 1], H = desc[5 * i + 2], pitch = desc[5 * i + 3];
    if (W < 1 || H < 1 || W > (1 << 20) || H > (1 << 20)) return fail(MRW_ERR_SHAPE, "instance %lld: bad size", (long long)i);
    if (off < 0 || off % 16 || pitch % 16 || pitch < W || pitch > INT32_MAX)
      return fail(MRW_ERR_CONSTRAINT, "instance %lld: offset and pitch must be multiples of 16, pitch >= W",
                  (long long)i);
    // H * pitch < 2^51 cannot overflow; off is compared on its own first
    if (off > arena_bytes || H * pitch > arena_bytes - off)
      return fail(MRW_ERR_SHAPE, "instance %lld lies outside the arena", (long long)i);
  }
  {
    // a captured call would leave graph nodes that read the shared host staging tables when the
    // graph is replayed, after later calls have overwritten them
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing((cudaStream_t)stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(MRW_ERR_UNSUPPORTED, "the allocation-free batched call cannot be captured into a CUDA graph");
  }
  mrw_config c = cfg ? *cfg : default_config(F_IMAGE);
  TRY(check_config(c));
  if (c.fusion != MRW_FUSE_ALL)
    return fail(MRW_ERR_UNSUPPORTED, "kernel-per-stage execution needs intermediate arenas; use mrw_execute_batched");
  ImgStage st[MRW_MAX_STAGES];
  int cnt = 0;
  TRY(collect_image_stages(root, st, &cnt, MRW_MAX_STAGES, 0));
  int blur_at = -1;
  for (int i = 0; i < cnt; ++i) {
    if (st[i].kind != OP_BLUR) continue;
    if (blur_at >= 0) return fail(MRW_ERR_UNSUPPORTED, "the allocation-free batched call fuses at most one blur");
    blur_at = i;
  }
  const int npre = blur_at >= 0 ? blur_at : cnt, nsuf = blur_at >= 0 ? cnt - blur_at - 1 : 0;
  if (npre > kMaxChainOps || nsuf > kMaxChainOps)
    return fail(MRW_ERR_UNSUPPORTED, "more than %d pointwise stages on one side of the blur", kMaxChainOps);
  StencilArgs a{};
  a.wait_polls = test_wait_polls();
  a.halo = blur_at >= 0 ? 2 : 0;
  a.npre = npre;
  a.nsuf = nsuf;
  fill_ops_array(st, npre, a.pre, &a.mpre);
  fill_ops_array(st + npre + (blur_at >= 0 ? 1 : 0), nsuf, a.suf, &a.msuf);
  const StencilShape s = stencil_shape(c, a);
  apply_shape(a, s);
  int dev = 0, sms = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const cudaError_t e =
      launch_stencil_noalloc(a, in_arena, out_arena, desc, n, sms, s.cps, s.smem, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "allocation-free batched launch");
  return MRW_OK;
}

extern "C" mrw_status mrw_noalloc_status(void *stream, uint32_t *host_status) {
  if (!host_status) return fail(MRW_ERR_INVALID_ARG, "host_status is NULL");
  unsigned int v = 0;
  const cudaError_t e = stencil_noalloc_status((cudaStream_t)stream, &v);
  if (e != cudaSuccess) return cuda_fail(e, "status of the allocation-free batched call");
  *host_status = v;
  if (v) return fail(MRW_ERR_DEVICE, "the last allocation-free batched call gave up a tile wait (status %u)", v);
  return MRW_OK;
}

// ============================================================================================
// CPU + GPU co-execution of a pointwise image tree (Section 3.3; the balancer is in coexec.cpp)
// ============================================================================================
namespace mrw {
mrw_status report_error(mrw_status s, const char *msg) {
  t_err = msg;
  return s;
}
}  // namespace mrw

extern "C" mrw_status mrw_execute_coexec(mrw_balancer_t b, mrw_node_t root, const mrw_buffer *args, int32_t nargs,
                                         const mrw_config *cfg, void *stream, mrw_balance_report *rep) {
  if (!b) return fail(MRW_ERR_INVALID_ARG, "balancer is NULL");
  if (nargs < 0 || (nargs && !args)) return fail(MRW_ERR_INVALID_ARG, "bad argument list");
  Program p;
  TRY(get_program(root, &p));
  if (p.fam != F_IMAGE || p.while_begin >= 0)
    return fail(MRW_ERR_UNSUPPORTED, "co-execution runs image trees without WHILE_CHANGED loops");
  if (nargs < 2 || args[0].memory != MRW_MEM_HOST || args[1].memory != MRW_MEM_HOST)
    return fail(MRW_ERR_UNSUPPORTED, "co-execution shares host image buffers between the GPU and the host cores");
  View vin, vout, vred;
  TRY(validate_image_args(p, args, nargs, &vin, &vout, &vred));
  const std::vector<Group> gs = group_stages(p, true, false);
  if (gs.size() != 1 || gs[0].use_stencil || gs[0].user || gs[0].reduce_only)
    return fail(MRW_ERR_UNSUPPORTED, "co-execution runs trees that fuse into one pointwise kernel");
  if (cfg) TRY(check_config(*cfg));
  HostChainOp ops[MRW_MAX_STAGES];
  int nops = 0;
  for (const ImgStage &s : p.img) {
    if (s.kind != OP_NOISE && s.kind != OP_SOLARISE && s.kind != OP_MIRROR && s.kind != OP_THRESH)
      return fail(MRW_ERR_UNSUPPORTED, "co-execution runs the built-in pointwise stages");
    ops[nops++] = HostChainOp{s.kind, s.seed, s.t};
  }
  const ImgGeom geo = geom_of(args[0], vin);
  std::lock_guard<std::mutex> lk(balancer_mutex(b));  // one co-executed run at a time per balancer
  const double share = balancer_share_locked(b);
  const int64_t gr = std::min<int64_t>(geo.rows, std::max<int64_t>(0, std::llround(share * (double)geo.rows)));
  const int64_t cr = geo.rows - gr;
  // the GPU's share: the first gr rows, as a (gr, W) image over the same host rows (the noise hash's
  // rows are global, and these are rows 0 .. gr-1); its MapReduce result stays in its future
  mrw_future_t fut = nullptr;
  if (gr > 0) {
    mrw_buffer sub[2] = {args[0], args[1]};
    const View *vv[2] = {&vin, &vout};
    for (int k = 0; k < 2; ++k) {
      sub[k].ndim = 2;
      sub[k].shape[0] = gr;
      sub[k].shape[1] = geo.W;
      sub[k].shape[2] = sub[k].shape[3] = 0;
      sub[k].pitch = vv[k]->pitch;
      sub[k].epu = 0;
    }
    TRY(execute(root, sub, 2, cfg, stream, &fut, true));
  }
  // the host threads' share, at the same time: rows gr .. rows-1
  const auto t0 = std::chrono::steady_clock::now();
  uint64_t cpu_red[3] = {0, 0, 0};
  if (cr > 0) {
    const mrw_status s = balancer_run_host_share(b, ops, nops, (const uint8_t *)args[0].data + gr * vin.pitch,
                                                 vin.pitch, (uint8_t *)args[1].data + gr * vout.pitch, vout.pitch,
                                                 (int)geo.W, gr, cr, p.reduce);
    if (s == MRW_OK) balancer_wait_host_share(b, cpu_red);
  }
  const double cpu_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  double gpu_ms = 0.0;
  int64_t gpu_red[3] = {0, 0, 0};
  if (fut) {
    mrw_status s = mrw_future_wait(fut, -1);
    float ms = 0.f;
    if (s == MRW_OK) s = mrw_future_elapsed_ms(fut, &ms);
    if (s == MRW_OK && p.reduce != RED_NONE)
      s = mrw_future_result(fut, gpu_red, sizeof(int64_t) * (p.reduce == RED_COUNT3 ? 3 : 1));
    const std::string msg = t_err;
    mrw_future_release(fut);
    if (s != MRW_OK) return fail(s, "%s", msg.c_str());
    gpu_ms = ms;
  }
  if (p.reduce != RED_NONE) {  // merging function + of the two partial results (Section 3.4)
    const int k = p.reduce == RED_COUNT3 ? 3 : 1;
    int64_t total[3];
    for (int i = 0; i < k; ++i) total[i] = gpu_red[i] + (int64_t)cpu_red[i];
    if (args[2].memory == MRW_MEM_HOST) {
      memcpy(args[2].data, total, sizeof(int64_t) * k);
    } else {
      CU(cudaMemcpyAsync(args[2].data, total, sizeof(int64_t) * k, cudaMemcpyHostToDevice, (cudaStream_t)stream));
      CU(cudaStreamSynchronize((cudaStream_t)stream));
    }
  }
  mrw_balance_report r{};
  balancer_observe_locked(b, gpu_ms, cpu_ms, &r);
  r.gpu_rows = gr;
  r.cpu_rows = cr;
  if (rep) *rep = r;
  return MRW_OK;
}
