#!/usr/bin/env python
"""Benchmark of the GB300 skeleton executor.

Headline workload (one "step" = one execution of the skeleton on one input):
  Map + MapReduce segmentation of a 512^3 uint8 volume (3-component mixture): the Map thresholds
  into 3 classes written as uint8 labels, the MapReduce (+) produces int64 class counts (Section 4
  of the paper, Segmentation). Algorithmic bytes per step: 128 MiB read + 128 MiB written + 24 B.
  value = fused skeleton GB/s over all ranks; the kernel-per-stage version is timed beside it.
Also measured in the same run (keys under "workloads"): the Filter Pipeline on 1024^2 and 8192^2,
N-body (65536 bodies, 100 Loop iterations, GFLOP/s at 20 flop per interaction), and the batched
4096-instance Filter Pipeline + 5x5 blur; each fused and kernel-per-stage.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mrw|reference] [--no-extras]
Under torchrun each rank runs its own replica on its own GPU (weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused skeleton GB/s & % HBM peak vs kernel-per-stage; N-body GFLOP/s"
SEG_SHAPE = (512, 512, 512)
SEG_BYTES = 2 * 512 ** 3 + 24
WORKLOAD = "segmentation 512^3 u8: Map(threshold 85/170 -> labels) + MapReduce(+) int64 class counts"


# --------------------------------------------------------------------------------------------
# clocks during the timed region (NVML through ctypes; read-only queries)
# --------------------------------------------------------------------------------------------
REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, device: int):
        self.samples = []
        self.max_mhz = None
        self.ok = False
        self._stop = threading.Event()
        try:
            import torch
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
            if self.nvml.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
                if self.nvml.nvmlDeviceGetHandleByIndex_v2(device, ctypes.byref(self.h)) != 0:
                    return
            m = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(m)) == 0:
                self.max_mhz = m.value
            self.reason_fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(self.nvml, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.ok = True
        except Exception:
            self.ok = False

    def sample(self):
        c = ctypes.c_uint()
        r = ctypes.c_ulonglong()
        if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0 and \
                self.reason_fn(self.h, ctypes.byref(r)) == 0:
            self.samples.append((c.value, r.value))

    def _run(self):
        while not self._stop.is_set():
            self.sample()
            time.sleep(0.002)

    def start(self):
        if self.ok:
            self.sample()
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()

    def stop(self):
        if self.ok:
            self._stop.set()
            self._t.join()
            self.sample()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"]}
        mhz = [s[0] for s in self.samples]
        bits = 0
        for s in self.samples:
            bits |= s[1]
        names = [n for b, n in REASONS.items() if bits & b and b != 0x1]
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": self.max_mhz, "reasons": names,
                "samples": len(self.samples), "source": "nvml"}


# --------------------------------------------------------------------------------------------
# distributed helpers (one process per GPU; barrier + max over ranks)
# --------------------------------------------------------------------------------------------
def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def recorded_traffic(kernel_src: str, key: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(key)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_1510_06585_gb300", "csrc", kernel_src)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec["dram_bytes"] if rec.get("source_sha256_16") == h else None


# --------------------------------------------------------------------------------------------
# timing helpers
# --------------------------------------------------------------------------------------------
def time_steps(fn, steps, warmup, world, device, sampler=None):
    """Run warmup then exactly `steps` timed calls of fn(i); returns (max-over-ranks seconds)."""
    import torch
    for i in range(warmup):
        fn(i)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
    e0.record(s)
    h0 = time.perf_counter()
    for i in range(steps):
        fn(i)
    time_steps.host_enqueue_us = (time.perf_counter() - h0) / max(steps, 1) * 1e6
    e1.record(s)
    torch.cuda.synchronize()
    if sampler:
        sampler.stop()
    barrier(world)
    torch.cuda.synchronize()
    return max_over_ranks(e0.elapsed_time(e1) / 1e3, world, device)


def tune_candidates(M, tree, args, reps=15, passes=2):
    """Time the 16 candidate configurations; return (best fused, best kernel-per-stage, summary).
    Each pass times every candidate (median of `reps` runs); a candidate keeps its best pass, so
    that a drift of the clock during one pass does not decide between candidates a few per cent
    apart."""
    cfgs = M.tune_candidates(tree, args)
    t = np.min(np.stack([np.asarray(M.tune_measure(tree, args, cfgs, reps=reps)) for _ in range(passes)]), axis=0)
    fused = [i for i in range(len(cfgs)) if cfgs[i].fusion == M.MRW_FUSE_ALL and t[i] > 0]
    unfused = [i for i in range(len(cfgs)) if cfgs[i].fusion == M.MRW_FUSE_NONE and t[i] > 0]
    bf = min(fused, key=lambda i: t[i])
    bu = min(unfused, key=lambda i: t[i])
    return cfgs[bf], cfgs[bu], {"fused_index": bf, "fused_cfg": list(cfgs[bf].as_tuple()),
                                "unfused_index": bu, "default_ms": round(float(t[0]), 5),
                                "best_ms": round(float(t[bf]), 5), "candidates": 16}


def run_mrw(args):
    import torch

    from paper_1510_06585_gb300 import inputs
    from paper_1510_06585_gb300 import mrw as M

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    # all work of the run, timed or not, goes to one stream of its own: launches into the legacy
    # default stream cost the host more (its implicit synchronisation with other streams)
    torch.cuda.set_stream(torch.cuda.Stream(device))
    M.load()
    peaks, peak_src = load_peaks()
    K, W = args.steps, args.warmup

    if not args.segmentation:  # profiling runs of one extra workload only
        lib = M.load()
        pending = []

        def drain_only():
            for fut in pending:
                s = lib.mrw_future_wait(fut, -1)
                lib.mrw_future_release(fut)
                M.check(s, "future")
            pending.clear()

        out = extras(M, lib, device, world, torch.cuda.current_stream().cuda_stream, peaks, pending, drain_only,
                     set(args.workloads.split(",")), args.batch_n, args.filter_sides)
        if rank == 0:
            print(json.dumps({"workloads": out}), flush=True)
        return

    # ---------------- headline: fused Map + MapReduce segmentation ----------------
    vol = inputs.volume(*SEG_SHAPE)
    sets = []
    for _ in range(2):  # two input/output sets: 512 MiB in flight, > 2x the 129 MB L2
        x = torch.from_numpy(vol).to(device)
        y = torch.empty_like(x)
        c = torch.zeros(3, dtype=torch.int64, device=device)
        sets.append((x, y, c))
    tree = M.mapreduce(M.map_(M.stage("threshold3")))
    lib = M.load()
    bufs = [M.buffers(*s) for s in sets]
    stream = torch.cuda.current_stream().cuda_stream

    # futures are released after the timed region (releasing one waits for its work)
    pending = []

    def step_async(cfg):
        run, h, cfgp = lib.mrw_execute, tree.h, ctypes.byref(cfg)

        def f(i):
            fut = ctypes.c_void_p()
            rc = run(h, bufs[i & 1], 3, cfgp, stream, ctypes.byref(fut))
            if rc:
                M.check(rc, "execute")
            pending.append(fut)
        return f

    def drain():
        for fut in pending:
            s = lib.mrw_future_wait(fut, -1)
            lib.mrw_future_release(fut)
            M.check(s, "future")
        pending.clear()

    # the executor's autotuner picks the launch configuration (all 16 candidates timed on these
    # buffers); the kernel-per-stage baseline gets the best of its own 8 candidates
    if args.fused_cfg:  # profiling runs: a given fused shape, no tuner launches before it
        blk, cps, tr, tc, un = (int(v) for v in args.fused_cfg.split(","))
        fused_cfg = M.config(block=blk, ctas_per_sm=cps, tile_rows=tr, tile_cols=tc, unroll=un)
        unfused_cfg = M.config(fusion=M.MRW_FUSE_NONE)
        tuning = {"fused_cfg": list(fused_cfg.as_tuple()), "note": "given with --fused-cfg (no tuning)"}
    else:
        fused_cfg, unfused_cfg, tuning = tune_candidates(M, tree, list(sets[0]))
    # kernels one step launches: each group's kernel, plus the one-CTA finish of a MapReduce group
    plan = M.plan_describe(tree, list(sets[0]), fused_cfg)
    launches_per_step = sum(1 + bool(g.get("finish_kernel")) for g in plan["groups"])
    sampler = ClockSampler(local)
    t_fused = time_steps(step_async(fused_cfg), K, W, world, device, sampler)
    host_enqueue_us = time_steps.host_enqueue_us  # host time to enqueue one step (no GPU wait inside)
    drain()
    # correctness of what was timed
    hist = np.bincount(np.digitize(vol.reshape(-1), [85, 170]), minlength=3).astype(np.int64)
    for x, y, c in sets:
        assert np.array_equal(c.cpu().numpy(), hist), "segmentation counts differ from the histogram"
    t_unfused = time_steps(step_async(unfused_cfg), K, W, world, device)
    drain()
    # the same bytes moved by a plain device copy (torch's copy kernel, 128 MiB read + 128 MiB
    # written per step over the same two rotating sets): what one launch of this size can reach
    def copy_step(i):
        x, y, _ = sets[i & 1]
        y.copy_(x)
    t_copy = time_steps(copy_step, K, W, world, device) / K
    fused_s = t_fused / K
    unfused_s = t_unfused / K
    value = world * SEG_BYTES * K / t_fused / 1e9

    # ---------------- e2e: host buffers through the C ABI ----------------
    hx = torch.from_numpy(vol).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    hc = torch.zeros(3, dtype=torch.int64).pin_memory()
    hbuf = M.buffers(hx, hy, hc)

    def e2e_with(cfg):
        def e2e_step(i):
            fut = ctypes.c_void_p()
            M.check(lib.mrw_execute(tree.h, hbuf, 3, ctypes.byref(cfg), stream, ctypes.byref(fut)), "execute")
            pending.append(fut)
        return e2e_step

    # the launch shape that suits HBM need not suit the host link: pick the end-to-end run's own
    # among the fused candidates, by a few timed steps each on these host buffers
    e2e_cands = [c for c in M.tune_candidates(tree, list(sets[0])) if c.fusion == M.MRW_FUSE_ALL]
    e2e_t = []
    for c in e2e_cands:
        e2e_t.append(time_steps(e2e_with(c), 4, 1, world, device))
        drain()
    e2e_cfg = e2e_cands[int(np.argmin(e2e_t))]
    k_e2e = max(1, min(K, 50))
    t_e2e = time_steps(e2e_with(e2e_cfg), k_e2e, min(W, 3), world, device)
    drain()
    assert np.array_equal(hc.numpy(), hist)
    e2e_value = world * SEG_BYTES * k_e2e / t_e2e / 1e9

    # what the host link carries: the copy engines moving the same bytes both ways at once (the
    # input to the device on one stream, the device labels back on another), 128 MiB each way
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    dx_, dy_ = sets[0][0], sets[1][1]

    def link_step(i):
        cur = torch.cuda.current_stream()
        s_in.wait_stream(cur)
        s_out.wait_stream(cur)
        with torch.cuda.stream(s_in):
            dx_.copy_(hx, non_blocking=True)
        with torch.cuda.stream(s_out):
            hy.copy_(dy_, non_blocking=True)
        cur.wait_stream(s_in)
        cur.wait_stream(s_out)
    k_link = max(1, min(K, 20))
    t_link = time_steps(link_step, k_link, min(W, 3), world, device)
    link_gbs = world * 2 * 512 ** 3 * k_link / t_link / 1e9

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(fused_s * 1e3, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic (seeded 3-component mixture volume)",
        "config": {"workload": WORKLOAD, "shape": list(SEG_SHAPE), "l2": "2 rotating input/output sets, 512 MiB > 2x L2",
                   "parallelism": f"replicas x{world}", "launch": "fused chain kernel, autotuned config",
                   "tuned": tuning},
        "kernel_per_stage": {"value": round(world * SEG_BYTES * K / t_unfused / 1e9, 2), "unit": "GB/s",
                             "ms_per_step": round(unfused_s * 1e3, 5),
                             "speedup_fused": round(unfused_s / fused_s, 3)},
        "roofline": {"bound": "hbm", "achieved": round(SEG_BYTES / fused_s / 1e9, 2), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(SEG_BYTES / fused_s / 1e9 / peaks["hbm_gbs"], 4),
                     "traffic": recorded_traffic("k_chain.cu", "segmentation_512cubed_chain"),
                     "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                     "copy_same_size_gbs": round(2 * 512 ** 3 / t_copy / 1e9, 2),
                     "frac_of_copy_same_size": round((2 * 512 ** 3 / fused_s) / (2 * 512 ** 3 / t_copy), 4),
                     "note": "achieved = algorithmic bytes / CUDA-event time of the step (the chain kernel and the "
                             "one-CTA MapReduce finish kernel behind it)"},
        "e2e": {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": 512 ** 3,
                "d2h_bytes_per_step": 512 ** 3 + 24, "steps": k_e2e,
                "host_link_copy_gbs": round(link_gbs, 2), "frac_of_host_link": round(e2e_value / link_gbs, 4),
                "cfg": list(e2e_cfg.as_tuple()),
                "note": "pinned host buffers read and written in place over NVLink-C2C by the fused kernel; "
                        "host_link_copy_gbs = the copy engines moving the same bytes both ways at once"},
        "gpu_launches": K * launches_per_step,
        "host_enqueue_us_per_step": round(host_enqueue_us, 2),
        "clocks": sampler.summary(),
    }

    # ---------------- other workloads of the hot path ----------------
    if args.extras:
        result["workloads"] = extras(M, lib, device, world, stream, peaks, pending, drain,
                                     set(args.workloads.split(",")), args.batch_n, args.filter_sides)

    # ---------------- CPU baseline (oracle) ----------------
    if rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(vol)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def tune_candidates_buffers(M, tree, bufarr, reps=5):
    """tune_candidates on a prepared mrw_buffer array."""
    lib = M.load()
    n = len(bufarr)
    cnt = ctypes.c_int32()
    M.check(lib.mrw_tune_candidates(tree.h, bufarr, n, None, 0, ctypes.byref(cnt)), "candidates")
    cfgs = (M.mrw_config * cnt.value)()
    M.check(lib.mrw_tune_candidates(tree.h, bufarr, n, cfgs, cnt.value, ctypes.byref(cnt)), "candidates")
    t = (ctypes.c_float * cnt.value)()
    M.check(lib.mrw_tune_measure(tree.h, bufarr, n, cfgs, cnt.value, reps,
                                 M.stream_handle(), t), "measure")
    t = np.array(t[:])
    fused = [i for i in range(cnt.value) if cfgs[i].fusion == M.MRW_FUSE_ALL and t[i] > 0]
    unfused = [i for i in range(cnt.value) if cfgs[i].fusion == M.MRW_FUSE_NONE and t[i] > 0]
    bf = min(fused, key=lambda i: t[i])
    bu = min(unfused, key=lambda i: t[i])
    return cfgs[bf], cfgs[bu], {"fused_index": bf, "fused_cfg": list(cfgs[bf].as_tuple()), "unfused_index": bu,
                                "default_ms": round(float(t[0]), 5), "best_ms": round(float(t[bf]), 5)}


def extras(M, lib, device, world, stream, peaks, pending, drain, which, batch_n, filter_sides="1024,4096,8192,16384"):
    import torch

    from paper_1510_06585_gb300 import inputs
    out = {}

    def timed(fn, reps, warm=2):
        for i in range(warm):
            fn(i)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(reps):
            fn(i)
        e1.record()
        torch.cuda.synchronize()
        drain()
        return e0.elapsed_time(e1) / 1e3 / reps

    def launcher(tree, bufsets, cfg):
        run, h, cfgp, nargs, nsets = lib.mrw_execute, tree.h, ctypes.byref(cfg), len(bufsets[0]), len(bufsets)

        def f(i):
            fut = ctypes.c_void_p()
            rc = run(h, bufsets[i % nsets], nargs, cfgp, stream, ctypes.byref(fut))
            if rc:
                M.check(rc, "execute")
            pending.append(fut)
        return f

    fused, unfused = M.config(), M.config(fusion=M.MRW_FUSE_NONE)
    # Filter Pipeline (noise -> solarise -> mirror)
    ftree = M.pipeline(M.stage("noise", seed=2), M.stage("solarise"), M.stage("mirror"))
    sides = [int(v) for v in filter_sides.split(",") if v] if "filter" in which else []
    # sides up to 2048 are L2-resident (reported as latency); above, enough rotating input/output
    # sets that consecutive steps touch at least 512 MiB (about 4x L2), at least two sets
    for side, nsets in ((v, 1 if v <= 2048 else max(2, -(-(512 << 20) // (2 * v * v)))) for v in sides):
        img = inputs.filter_image(side, side)
        sets = []
        for _ in range(nsets):
            x = torch.from_numpy(img).to(device)
            sets.append(M.buffers(x, torch.empty_like(x)))
        reps = 200 if side == 1024 else 20
        f_cfg, u_cfg, tinfo = tune_candidates_buffers(M, ftree, sets[0])
        tf = timed(launcher(ftree, sets, f_cfg), reps)
        tu = timed(launcher(ftree, sets, u_cfg), reps)
        b = 2 * side * side
        out[f"filter_{side}"] = {"fused_gbs": round(b / tf / 1e9, 1), "fused_us": round(tf * 1e6, 2), "tuned": tinfo,
                                 "kernel_per_stage_gbs": round(b / tu / 1e9, 1), "speedup_fused": round(tu / tf, 3),
                                 "frac_hbm": round(b / tf / 1e9 / peaks["hbm_gbs"], 4),
                                 "l2": (f"resident ({b >> 20} MiB)" if nsets == 1 and side <= 2048 else
                                        f"{nsets} rotating sets, {nsets * b >> 20} MiB")}
    if "nbody" in which:
        out.update(nbody_workload(M, device, timed, launcher, fused, unfused))
    if "batched" in which:
        out.update(batched_workload(M, lib, device, timed, pending, fused, unfused, peaks, stream, batch_n))
    if "fft" in which:
        out.update(fft_workload(M, device, timed, launcher, fused, unfused, peaks))
    if "costmodel" in which:
        out.update(costmodel_workload())
    return out


def fft_workload(M, device, timed, launcher, fused, unfused, peaks, nfft=256):
    """FFT pipelined with its inversion (Section 4): 256 rows of 65536 complex float32 values
    (one 512 KB elementary unit each, 128 MB in total); forward then inverse transform of every
    row, fused on chip (one cluster launch) and kernel per stage (two launches through HBM)."""
    import torch

    from paper_1510_06585_gb300 import inputs
    n = 65536
    x = torch.from_numpy(inputs.fft_signals(nfft, n)).to(device)
    y = torch.empty_like(x)
    tree = M.pipeline(M.stage("fft"), M.stage("ifft"))
    sets = [M.buffers(x, y)]
    tf = timed(launcher(tree, sets, fused), 20)
    tu = timed(launcher(tree, sets, unfused), 20)
    b = 2 * nfft * n * 8                      # read the input once, write the output once
    flop = 2 * 5.0 * n * 16 * nfft            # 5 N log2 N per transform, two transforms
    return {f"fft_ifft_{nfft}x65536": {"fused_gbs": round(b / tf / 1e9, 1), "fused_us": round(tf * 1e6, 1),
                                       "gflops": round(flop / tf / 1e9, 1),
                                       "kernel_per_stage_gbs": round(b / tu / 1e9, 1),
                                       "speedup_fused": round(tu / tf, 3),
                                       "frac_hbm": round(b / tf / 1e9 / peaks["hbm_gbs"], 4),
                                       "bytes": b, "l2": "128 MB in + 128 MB out per step (> L2)"}}


def costmodel_workload(n_train=4000, n_test=500, max_log2=26):
    """Learned configuration derivation on random compound skeletons: the MLP (the library's own
    bf16/fp32 forward, backward and Adam kernels) is trained on the exhaustive tuner's timings and
    its choices on unseen skeletons are scored by regret against the tuner's best."""
    from paper_1510_06585_gb300 import costmodel as C
    t0 = time.perf_counter()
    res, _, _ = C.experiment(n_train, n_test, max_log2=max_log2, epochs=300, reps=3, log=None)
    r = lambda d: {k: round(v, 4) for k, v in d.items()}
    return {"costmodel": {"n_train": n_train, "n_test": n_test, "max_log2": max_log2,
                          "regret_learned": r(res["learned"]), "regret_default": r(res["default_config"]),
                          "regret_nearest_neighbour": r(res["nearest_neighbour_kb"]),
                          "train_seconds": res["train_seconds"], "seconds": round(time.perf_counter() - t0, 1)}}


def nbody_workload(M, device, timed, launcher, fused, unfused):
    import torch

    from paper_1510_06585_gb300 import inputs
    out = {}
    # N-body: accel + Loop(100 KDK)
    n = 65536
    xs, vs, as_ = inputs.nbody(n)
    st = [torch.from_numpy(t).to(device) for t in (xs, vs, as_)]
    kdk = M.stage("nbody_kdk", eps=1e-3, dt=1e-3)
    ntree = M.pipeline(M.stage("nbody_accel", eps=1e-3, dt=1e-3), M.loop(kdk, 100))
    nb = [M.buffers(*st)]
    tn = timed(launcher(ntree, nb, fused), 3, warm=1)
    tnu = timed(launcher(ntree, nb, unfused), 1, warm=0)
    inter = float(n) * n * 101
    alu_peak = 20.0 * 152 * 128 * 2070e6 / 12 / 1e9  # GFLOP/s at 12 FP32-pipe instructions per interaction
    gf = 20.0 * inter / tn / 1e9
    out["nbody_65536x100"] = {"gflops": round(gf, 1), "ms": round(tn * 1e3, 2),
                              "interactions_per_s": round(inter / tn, 1),
                              "frac_alu": round(gf / alu_peak, 4), "alu_peak_gflops": round(alu_peak, 1),
                              "kernel_per_step_host_loop_ms": round(tnu * 1e3, 2),
                              "speedup_fused": round(tnu / tn, 3)}
    return out


def batched_workload(M, lib, device, timed, pending, fused, unfused, peaks, stream, batch_n):
    import torch

    from paper_1510_06585_gb300 import inputs
    out = {}
    # Batched: instances of Filter Pipeline + 5x5 blur, sides log-uniform in 64..2048
    shapes = inputs.batch_shapes(batch_n)
    desc, nbytes = inputs.batch_descriptors(shapes)
    arena = inputs.batch_arena(desc, nbytes)
    bx = torch.from_numpy(arena).to(device)
    by = torch.zeros_like(bx)
    btree = M.map_(M.pipeline(M.stage("noise"), M.stage("solarise"), M.stage("mirror"), M.stage("blur5")))
    d = np.ascontiguousarray(desc, dtype=np.int64)
    dptr = d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))

    def blaunch(cfg, tree=btree):
        def f(i):
            fut = ctypes.c_void_p()
            M.check(lib.mrw_execute_batched(tree.h, bx.data_ptr(), by.data_ptr(), bx.numel(), dptr, d.shape[0],
                                            ctypes.byref(cfg), stream, ctypes.byref(fut)), "batched")
            pending.append(fut)
        return f

    px = float((shapes[:, 0] * shapes[:, 1]).sum())
    # autotune the batched launch over the candidate tile shapes (fused and kernel-per-stage)
    cand = M.tune_candidates(btree, [bx[:64].view(8, 8), by[:64].view(8, 8)])
    times = [timed(blaunch(c), 2, warm=1) for c in cand]
    bf = min(range(8), key=lambda i: times[i])
    bu = min(range(8, 16), key=lambda i: times[i])
    tb = timed(blaunch(cand[bf]), 5)
    tbu = timed(blaunch(cand[bu]), 3)
    # where the time goes: the same batch and launch shape with the leading stages removed
    subsets = {}
    for names in (["blur5"], ["mirror", "blur5"], ["solarise", "mirror", "blur5"]):
        sub = M.map_(M.pipeline(*[M.stage(nm) for nm in names]))
        subsets["+".join(names)] = round(timed(blaunch(cand[bf], sub), 3) * 1e3, 3)
    out[f"batched_{batch_n}"] = {"fused_gbs": round(2 * px / tb / 1e9, 1), "fused_ms": round(tb * 1e3, 3),
                           "pixels": int(px), "kernel_per_stage_gbs": round(2 * px / tbu / 1e9, 1),
                           "speedup_fused": round(tbu / tb, 3), "frac_hbm": round(2 * px / tb / 1e9 / peaks["hbm_gbs"], 4),
                           "launches_per_step": 1, "stage_subsets_ms": subsets,
                           "tuned": {"fused_index": bf, "fused_cfg": list(cand[bf].as_tuple()),
                                                             "unfused_index": bu,
                                                             "default_ms": round(times[0] * 1e3, 4)}}
    return out


def cpu_baseline(vol, min_seconds=8.0):
    """The oracle as it stands on a bounded sample of the workload (the first 128 planes)."""
    from oracle import image as O
    sample = vol[:128]
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < min_seconds:
        O.segmentation(sample)
        reps += 1
    dt = time.perf_counter() - t0
    b = (2 * sample.size + 24) * reps
    return {"value": round(b / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} x Map+MapReduce on the first 128 of 512 planes (32 MiB), numpy single thread",
            "seconds": round(dt, 2)}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import image as O
    from paper_1510_06585_gb300 import inputs
    sample = inputs.volume(32, 512, 512)  # a bounded sample of the workload per step (8 MiB)
    for _ in range(args.warmup):
        O.segmentation(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.segmentation(sample)
    dt = time.perf_counter() - t0
    b = (2 * sample.size + 24) * args.steps
    v = b / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded 3-component mixture volume)",
            "config": {"workload": WORKLOAD, "shape": list(SEG_SHAPE)},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: Map+MapReduce on 32 of the 512 planes (8 MiB in, 8 MiB of "
                                       "labels out), numpy single thread; GB/s = bytes of the sample / time"},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mrw", choices=["mrw", "reference"])
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--workloads", default="filter,nbody,batched,fft,costmodel",
                    help="comma list of the extra workloads to run (filter, nbody, batched, fft, costmodel)")
    ap.add_argument("--batch-n", type=int, default=4096, help="instances of the batched workload")
    ap.add_argument("--filter-sides", default="1024,4096,8192,16384", help="image sides of the Filter Pipeline workload")
    ap.add_argument("--fused-cfg", default="",
                    help="block,ctas_per_sm,tile_rows,tile_cols,unroll of the headline's fused launch "
                         "(profiling runs; default: the autotuner's choice)")
    ap.add_argument("--no-segmentation", dest="segmentation", action="store_false",
                    help="skip the headline timing (profiling runs of one extra workload)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mrw":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mrw(args)


if __name__ == "__main__":
    main()
