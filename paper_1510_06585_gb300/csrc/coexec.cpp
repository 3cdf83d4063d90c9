// CPU + GPU co-execution: the host worker threads' share of a pointwise image chain, and the
// balancer that decides the shares (Section 3.2, the workload distribution generator's binary
// search; Section 3.3, the load balancing threshold lbt and the adaptive binary search).
//
// On Grace + GB300 the host cores and the GPU both reach page-locked host memory (the GPU over
// NVLink-C2C), so a tree over host buffers can be split by rows: the GPU streams the first rows
// in place, the host threads compute the rest at the same time, and the partial MapReduce results
// are merged on the host. The balancer moves rows between the two until their times agree.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#if defined(__linux__)
#include <sched.h>
#endif

#include "mrw.h"
#include "mrw_internal.h"

namespace mrw {

// ------------------------------------------------------------------------------------------
// The host share of a pointwise chain: stage after stage on one row at a time
// ------------------------------------------------------------------------------------------
namespace {

// MurmurHash3's 32-bit finaliser (Appleby; public domain), as the noise stage defines it.
inline uint32_t fmix32_host(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// One row through the stages, in place in `row` (W pixels); y is the row's global index.
void chain_row(const HostChainOp *ops, int nops, uint8_t *row, int W, uint32_t y) {
  for (int i = 0; i < nops; ++i) {
    const HostChainOp &op = ops[i];
    switch (op.kind) {
      case OP_NOISE: {
        const uint32_t fs = fmix32_host(op.seed);
        for (int x = 0; x < W; ++x) {
          const uint32_t h = fmix32_host(fmix32_host(fs ^ (uint32_t)x) ^ y);
          const int v = (int)row[x] + (int)(h % 41u) - 20;
          row[x] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
        }
        break;
      }
      case OP_SOLARISE:
        for (int x = 0; x < W; ++x) row[x] = row[x] < 128 ? row[x] : (uint8_t)(255 - row[x]);
        break;
      case OP_MIRROR:
        std::reverse(row, row + W);
        break;
      case OP_THRESH: {
        const uint8_t t0 = (uint8_t)(op.t & 0xFF), t1 = (uint8_t)((op.t >> 8) & 0xFF);
        for (int x = 0; x < W; ++x) row[x] = (uint8_t)((row[x] >= t0) + (row[x] >= t1));
        break;
      }
      default:
        break;
    }
  }
}

}  // namespace

void host_chain_rows(const HostChainOp *ops, int nops, const uint8_t *in, int64_t in_pitch, uint8_t *out,
                     int64_t out_pitch, int W, int64_t y0, int64_t r0, int64_t r1, int reduce, uint64_t *red3) {
  std::vector<uint8_t> buf((size_t)W);
  uint64_t c[3] = {0, 0, 0};
  for (int64_t r = r0; r < r1; ++r) {
    memcpy(buf.data(), in + r * in_pitch, (size_t)W);
    chain_row(ops, nops, buf.data(), W, (uint32_t)(y0 + r));
    memcpy(out + r * out_pitch, buf.data(), (size_t)W);
    if (reduce == RED_COUNT3) {
      uint32_t n1 = 0, n2 = 0;  // labels are 0, 1, 2: count the ones and the twos
      for (int x = 0; x < W; ++x) {
        n1 += buf[x] == 1;
        n2 += buf[x] == 2;
      }
      c[1] += n1;
      c[2] += n2;
      c[0] += (uint64_t)W - n1 - n2;
    } else if (reduce == RED_SUM) {
      uint64_t s = 0;
      for (int x = 0; x < W; ++x) s += buf[x];
      c[0] += s;
    }
  }
  for (int k = 0; k < 3; ++k) red3[k] = c[k];
}

// ------------------------------------------------------------------------------------------
// Worker threads: a job is a number of blocks, taken one at a time by the threads
// ------------------------------------------------------------------------------------------
class WorkerPool {
 public:
  explicit WorkerPool(int n) {
    for (int i = 0; i < n; ++i) threads_.emplace_back([this] { loop(); });
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (std::thread &t : threads_) t.join();
  }
  int size() const { return (int)threads_.size(); }
  // Start fn(block) for block in [0, nblocks) on the workers; returns at once.
  void start(int64_t nblocks, std::function<void(int64_t)> fn) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = std::move(fn);
      nblocks_ = nblocks;
      next_.store(0);
      done_blocks_ = 0;
      ++gen_;
    }
    cv_.notify_all();
  }
  // Wait until every block of the started job has run.
  void wait() {
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [this] { return done_blocks_ >= nblocks_; });
  }

 private:
  void loop() {
    uint64_t seen = 0;
    while (true) {
      std::function<void(int64_t)> fn;
      int64_t nb = 0;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        fn = fn_;
        nb = nblocks_;
      }
      int64_t ran = 0;
      for (int64_t b = next_.fetch_add(1); b < nb; b = next_.fetch_add(1)) {
        fn(b);
        ++ran;
      }
      if (ran) {
        std::lock_guard<std::mutex> lk(mu_);
        done_blocks_ += ran;
        if (done_blocks_ >= nblocks_) done_cv_.notify_all();
      }
    }
  }
  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::function<void(int64_t)> fn_;
  int64_t nblocks_ = 0, done_blocks_ = 0;
  std::atomic<int64_t> next_{0};
  uint64_t gen_ = 0;
  bool stop_ = false;
};

}  // namespace mrw

using namespace mrw;

// ------------------------------------------------------------------------------------------
// The balancer (Section 3.3)
// ------------------------------------------------------------------------------------------
struct mrw_balancer {
  mrw_balance_params prm{};
  std::mutex mu;
  // state
  int phase = MRW_BAL_SEARCH;
  double lbt = 0.0;
  double share = 0.5;    // GPU share of the next run
  double bound_gpu = 0.0, bound_cpu = 0.0;  // profile construction: work bound to each side
  double t = 1.0;        // transferable part
  int last_dir = 0;      // +1: the last move gave the GPU more work, -1: the host
  int same_dir = 0;      // consecutive moves in last_dir
  int reps_seen = 0;     // profile construction: runs observed at the current share
  double best_gpu = 0.0, best_cpu = 0.0;  // and the fastest time of each side among them
  std::unique_ptr<WorkerPool> pool;
  // per-run scratch of the host share's partial results
  std::vector<std::array<uint64_t, 3>> partial;
};

namespace {

int available_cores() {
#if defined(__linux__)
  cpu_set_t set;
  if (sched_getaffinity(0, sizeof set, &set) == 0) {
    const int n = CPU_COUNT(&set);
    if (n > 0) return n;
  }
#endif
  const unsigned n = std::thread::hardware_concurrency();
  return n ? (int)n : 1;
}

double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

// One run observed: deviation, lbt and the share of the next run.
void observe_locked(mrw_balancer *b, double gpu_ms, double cpu_ms, mrw_balance_report *rep) {
  const double ran_share = b->share;
  const double hi = std::max(gpu_ms, cpu_ms), lo = std::min(gpu_ms, cpu_ms);
  const double dev = hi > 0.0 ? lo / hi : 1.0;
  const int unbalanced = dev / b->prm.c_factor < b->prm.max_dev ? 1 : 0;
  b->lbt = unbalanced * b->prm.weight + b->lbt * (1.0 - b->prm.weight);
  // the faster side takes work: +1 moves rows to the GPU, -1 to the host threads
  const int dir = gpu_ms < cpu_ms ? +1 : -1;
  switch (b->phase) {
    case MRW_BAL_SEARCH: {
      // each share runs search_reps times; the fastest time of each side decides
      b->best_gpu = b->reps_seen ? std::min(b->best_gpu, gpu_ms) : gpu_ms;
      b->best_cpu = b->reps_seen ? std::min(b->best_cpu, cpu_ms) : cpu_ms;
      if (++b->reps_seen < b->prm.search_reps) break;
      const int sdir = b->best_gpu < b->best_cpu ? +1 : -1;
      b->reps_seen = 0;
      // the transferable part was split evenly; the faster side keeps its half for good
      const double half = b->t / 2.0;
      if (sdir > 0) b->bound_gpu += half;
      else b->bound_cpu += half;
      b->t = half;
      b->share = clamp01(b->bound_gpu + b->t / 2.0);
      if (b->t < b->prm.precision) {
        b->phase = MRW_BAL_MONITOR;
        b->lbt = 0.0;
      }
      break;
    }
    case MRW_BAL_MONITOR:
      if (b->lbt >= b->prm.trigger) {
        // a persistent imbalance: the adaptive binary search starts from a transferable part of
        // one sixteenth of the work and first shifts towards the faster side
        b->phase = MRW_BAL_SHIFT;
        b->t = std::max(b->prm.precision, 1.0 / 16.0);
        b->same_dir = 1;
        b->last_dir = dir;
        b->share = clamp01(b->share + dir * b->t);
      }
      break;
    case MRW_BAL_SHIFT:
    case MRW_BAL_BISECT: {
      if (dir != b->last_dir) {  // the balance point lies between the last two shares: halve
        b->phase = MRW_BAL_BISECT;
        b->t /= 2.0;
        b->same_dir = 1;
        b->last_dir = dir;
      } else if (++b->same_dir > 2) {  // more than two moves the same way: shift, and faster
        b->phase = MRW_BAL_SHIFT;
        b->t *= 2.0;
      } else if (b->phase == MRW_BAL_BISECT) {
        b->t /= 2.0;
      }
      b->t = std::min(b->t, 0.5);
      b->share = clamp01(b->share + dir * b->t);
      if (b->phase == MRW_BAL_BISECT && b->t < b->prm.precision) {
        b->phase = MRW_BAL_MONITOR;
        b->lbt = 0.0;
      }
      break;
    }
  }
  if (rep) {
    rep->gpu_share = ran_share;
    rep->gpu_ms = gpu_ms;
    rep->cpu_ms = cpu_ms;
    rep->dev = dev;
    rep->unbalanced = unbalanced;
    rep->phase = b->phase;
    rep->lbt = b->lbt;
    rep->next_share = b->share;
    rep->transferable = b->t;
  }
}

}  // namespace

namespace mrw {

mrw_status balancer_run_host_share(mrw_balancer *b, const HostChainOp *ops, int nops, const uint8_t *in,
                                   int64_t in_pitch, uint8_t *out, int64_t out_pitch, int W, int64_t y0,
                                   int64_t rows, int reduce) {
  const int64_t per = std::max<int64_t>(1, std::min<int64_t>(64, (1 << 20) / std::max(1, W)));
  const int64_t nblocks = (rows + per - 1) / per;
  b->partial.assign((size_t)nblocks, {0, 0, 0});
  if (nblocks == 0) return MRW_OK;
  std::vector<HostChainOp> op(ops, ops + nops);
  // runs after this function has returned: everything by value
  b->pool->start(nblocks, [=](int64_t k) {
    const int64_t r0 = k * per, r1 = std::min(rows, r0 + per);
    host_chain_rows(op.data(), (int)op.size(), in + r0 * in_pitch, in_pitch, out + r0 * out_pitch, out_pitch, W,
                    y0 + r0, 0, r1 - r0, reduce, b->partial[(size_t)k].data());
  });
  return MRW_OK;
}

void balancer_wait_host_share(mrw_balancer *b, uint64_t *red3) {
  b->pool->wait();
  red3[0] = red3[1] = red3[2] = 0;
  for (const auto &p : b->partial)
    for (int k = 0; k < 3; ++k) red3[k] += p[k];
}

double balancer_share_locked(mrw_balancer *b) { return b->share; }
std::mutex &balancer_mutex(mrw_balancer *b) { return b->mu; }
void balancer_observe_locked(mrw_balancer *b, double gpu_ms, double cpu_ms, mrw_balance_report *rep) {
  observe_locked(b, gpu_ms, cpu_ms, rep);
}

}  // namespace mrw

extern "C" {

mrw_status mrw_balancer_create(const mrw_balance_params *params, mrw_balancer_t *out) {
  if (!out) return report_error(MRW_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  mrw_balance_params p = params ? *params : mrw_balance_params{};
  if (p.weight == 0.0) p.weight = 2.0 / 3.0;
  if (p.max_dev == 0.0) p.max_dev = 0.85;
  if (p.c_factor == 0.0) p.c_factor = 1.0;
  if (p.trigger == 0.0) p.trigger = 0.95;
  if (p.precision == 0.0) p.precision = 1.0 / 256.0;
  if (p.search_reps == 0) p.search_reps = 1;
  const auto in01 = [](double v) { return v > 0.0 && v <= 1.0 && std::isfinite(v); };
  if (!in01(p.weight) || !in01(p.max_dev) || !in01(p.trigger) || !in01(p.precision) || !(p.c_factor > 0.0) ||
      !std::isfinite(p.c_factor) || !(p.gpu_share <= 1.0) || p.cpu_threads < 0 || p.search_reps < 1 ||
      p.search_reps > 64)
    return report_error(MRW_ERR_INVALID_ARG, "balancer parameter out of range");
  mrw_balancer *b = new (std::nothrow) mrw_balancer();
  if (!b) return report_error(MRW_ERR_OOM, "balancer");
  b->prm = p;
  if (p.gpu_share >= 0.0) {  // a converged profile: monitor from the given share
    b->phase = MRW_BAL_MONITOR;
    b->share = p.gpu_share;
    b->t = p.precision / 2.0;
  }
  try {
    b->pool.reset(new WorkerPool(p.cpu_threads ? p.cpu_threads : available_cores()));
  } catch (...) {
    delete b;
    return report_error(MRW_ERR_OOM, "balancer worker threads");
  }
  *out = b;
  return MRW_OK;
}

void mrw_balancer_release(mrw_balancer_t b) { delete b; }

mrw_status mrw_balancer_observe(mrw_balancer_t b, double gpu_ms, double cpu_ms, mrw_balance_report *rep) {
  if (!b || !(gpu_ms >= 0.0) || !(cpu_ms >= 0.0) || !std::isfinite(gpu_ms) || !std::isfinite(cpu_ms))
    return report_error(MRW_ERR_INVALID_ARG, "balancer NULL or a time negative or not finite");
  std::lock_guard<std::mutex> lk(b->mu);
  if (rep) *rep = mrw_balance_report{};
  observe_locked(b, gpu_ms, cpu_ms, rep);
  return MRW_OK;
}

mrw_status mrw_balancer_share(mrw_balancer_t b, double *gpu_share) {
  if (!b || !gpu_share) return report_error(MRW_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(b->mu);
  *gpu_share = b->share;
  return MRW_OK;
}

}  // extern "C"
