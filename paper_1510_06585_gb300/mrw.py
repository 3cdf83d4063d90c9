"""Thin Python binding of libmrw (include/mrw.h): the same names, argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only converts tensors and
numpy arrays into ``mrw_buffer`` descriptors and checks status codes. It never falls back to
another implementation: if libmrw.so cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MRW_OK = 0
MRW_ERR_INVALID_ARG, MRW_ERR_SHAPE, MRW_ERR_DTYPE, MRW_ERR_CONSTRAINT = 1, 2, 3, 4
MRW_ERR_OOM, MRW_ERR_CUDA, MRW_ERR_TIMEOUT, MRW_ERR_DEVICE, MRW_ERR_UNSUPPORTED, MRW_ERR_NOT_READY = 5, 6, 7, 8, 9, 10

MRW_U8, MRW_I32, MRW_I64, MRW_F32, MRW_F64, MRW_BF16, MRW_C64 = range(7)
MRW_MEM_DEVICE, MRW_MEM_HOST = 0, 1
MRW_PARTITION, MRW_COPY = 0, 1
(MRW_ST_NOISE_HASH, MRW_ST_SOLARISE, MRW_ST_MIRROR_H, MRW_ST_BOXBLUR5, MRW_ST_THRESHOLD3,
 MRW_ST_NBODY_ACCEL, MRW_ST_NBODY_KDK, MRW_ST_SAXPY, MRW_ST_FFT, MRW_ST_IFFT) = range(10)
MRW_RED_ADD, MRW_RED_SUB, MRW_RED_MUL, MRW_RED_DIV = range(4)
MRW_LOOP_FOR, MRW_LOOP_WHILE_CHANGED = 0, 1
MRW_FUSE_ALL, MRW_FUSE_NONE = 0, 1
MRW_TUNE_EXHAUSTIVE, MRW_TUNE_PRUNED, MRW_TUNE_MODEL = 0, 1, 2
MRW_NFEATURES = 16
MRW_NOALLOC_MAX_INSTANCES = 256

STAGE_BY_NAME = {"noise": MRW_ST_NOISE_HASH, "solarise": MRW_ST_SOLARISE, "mirror": MRW_ST_MIRROR_H,
                 "blur5": MRW_ST_BOXBLUR5, "threshold3": MRW_ST_THRESHOLD3, "nbody_accel": MRW_ST_NBODY_ACCEL,
                 "nbody_kdk": MRW_ST_NBODY_KDK, "saxpy": MRW_ST_SAXPY, "fft": MRW_ST_FFT, "ifft": MRW_ST_IFFT}


class mrw_buffer(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int), ("ndim", ctypes.c_int32),
                ("shape", ctypes.c_int64 * 4), ("pitch", ctypes.c_int64), ("epu", ctypes.c_int64),
                ("transfer", ctypes.c_int), ("memory", ctypes.c_int)]


class mrw_stage_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32), ("t0", ctypes.c_int32), ("t1", ctypes.c_int32), ("G", ctypes.c_float),
                ("eps", ctypes.c_float), ("dt", ctypes.c_float), ("alpha", ctypes.c_float), ("nu", ctypes.c_int32),
                ("wg", ctypes.c_int32)]


class mrw_loop_state(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int64), ("kind", ctypes.c_int32), ("global_sync", ctypes.c_int32)]


class mrw_config(ctypes.Structure):
    _fields_ = [("fusion", ctypes.c_int32), ("block", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32), ("tile_cols", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]

    def as_tuple(self):
        return (self.fusion, self.block, self.ctas_per_sm, self.tile_rows, self.tile_cols, self.unroll)


class mrw_balance_params(ctypes.Structure):
    _fields_ = [("weight", ctypes.c_double), ("max_dev", ctypes.c_double), ("c_factor", ctypes.c_double),
                ("trigger", ctypes.c_double), ("precision", ctypes.c_double), ("gpu_share", ctypes.c_double),
                ("cpu_threads", ctypes.c_int32), ("search_reps", ctypes.c_int32)]


class mrw_balance_report(ctypes.Structure):
    _fields_ = [("gpu_share", ctypes.c_double), ("gpu_rows", ctypes.c_int64), ("cpu_rows", ctypes.c_int64),
                ("gpu_ms", ctypes.c_double), ("cpu_ms", ctypes.c_double), ("dev", ctypes.c_double),
                ("unbalanced", ctypes.c_int32), ("phase", ctypes.c_int32), ("lbt", ctypes.c_double),
                ("next_share", ctypes.c_double), ("transferable", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


MRW_BAL_SEARCH, MRW_BAL_MONITOR, MRW_BAL_SHIFT, MRW_BAL_BISECT = range(4)

_P = ctypes.c_void_p
_SIGS = {
    "mrw_abi_version": (ctypes.c_int32, []),
    "mrw_last_error": (ctypes.c_char_p, []),
    "mrw_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mrw_stage": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(mrw_stage_params), ctypes.POINTER(_P)]),
    "mrw_stage_user": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.POINTER(_P)]),
    "mrw_pipeline_create": (ctypes.c_int, [ctypes.POINTER(_P)]),
    "mrw_pipeline_add_stage": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(mrw_stage_params)]),
    "mrw_pipeline_add_node": (ctypes.c_int, [_P, _P]),
    "mrw_map": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "mrw_mapreduce": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "mrw_loop": (ctypes.c_int, [_P, ctypes.POINTER(mrw_loop_state), ctypes.POINTER(_P)]),
    "mrw_node_retain": (None, [_P]),
    "mrw_node_release": (None, [_P]),
    "mrw_execute": (ctypes.c_int, [_P, ctypes.POINTER(mrw_buffer), ctypes.c_int32, ctypes.POINTER(mrw_config), _P,
                                   ctypes.POINTER(_P)]),
    "mrw_execute_timed": (ctypes.c_int, [_P, ctypes.POINTER(mrw_buffer), ctypes.c_int32, ctypes.POINTER(mrw_config),
                                         _P, ctypes.POINTER(_P)]),
    "mrw_execute_batched": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                           ctypes.POINTER(mrw_config), _P, ctypes.POINTER(_P)]),
    "mrw_execute_batched_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                                   ctypes.c_int64, ctypes.POINTER(mrw_config), _P]),
    "mrw_noalloc_status": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "mrw_future_wait": (ctypes.c_int, [_P, ctypes.c_int64]),
    "mrw_future_query": (ctypes.c_int, [_P]),
    "mrw_future_elapsed_ms": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "mrw_future_result": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "mrw_future_release": (None, [_P]),
    "mrw_fft_schedule_check": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_int64)]),
    "mrw_plan_describe": (ctypes.c_int, [_P, ctypes.POINTER(mrw_buffer), ctypes.c_int32, ctypes.POINTER(mrw_config),
                                         ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "mrw_tune_candidates": (ctypes.c_int, [_P, ctypes.POINTER(mrw_buffer), ctypes.c_int32, ctypes.POINTER(mrw_config),
                                           ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "mrw_tune_measure": (ctypes.c_int, [_P, ctypes.POINTER(mrw_buffer), ctypes.c_int32, ctypes.POINTER(mrw_config),
                                        ctypes.c_int32, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_float)]),
    "mrw_tune": (ctypes.c_int, [_P, ctypes.POINTER(mrw_buffer), ctypes.c_int32, ctypes.c_int, ctypes.c_int32, _P,
                                ctypes.POINTER(mrw_config), ctypes.POINTER(ctypes.c_float)]),
    "mrw_kb_save": (ctypes.c_int, [ctypes.c_char_p]),
    "mrw_kb_load": (ctypes.c_int, [ctypes.c_char_p]),
    "mrw_kb_clear": (ctypes.c_int, []),
    "mrw_kb_size": (ctypes.c_int64, []),
    "mrw_features": (ctypes.c_int, [_P, ctypes.POINTER(mrw_buffer), ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
    "mrw_model_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "mrw_model_release": (None, [_P]),
    "mrw_model_num_params": (ctypes.c_int64, [_P]),
    "mrw_model_set_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "mrw_model_get_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float)]),
    "mrw_model_forward": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "mrw_model_gradients": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_float), _P]),
    "mrw_model_adam_step": (ctypes.c_int, [_P, _P, ctypes.c_float, _P]),
    "mrw_model_train": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                       ctypes.c_uint64, _P, ctypes.POINTER(ctypes.c_float)]),
    "mrw_tune_set_model": (ctypes.c_int, [_P, ctypes.POINTER(mrw_config), ctypes.c_int32]),
    "mrw_balancer_create": (ctypes.c_int, [ctypes.POINTER(mrw_balance_params), ctypes.POINTER(_P)]),
    "mrw_balancer_release": (None, [_P]),
    "mrw_balancer_observe": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(mrw_balance_report)]),
    "mrw_balancer_share": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "mrw_execute_coexec": (ctypes.c_int, [_P, _P, ctypes.POINTER(mrw_buffer), ctypes.c_int32,
                                          ctypes.POINTER(mrw_config), _P, ctypes.POINTER(mrw_balance_report)]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmrw.so (building it first if needed) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libmrw.so is missing at {path}; run paper_1510_06585_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MrwError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.mrw_last_error().decode() if _lib else ""
        super().__init__(f"{where}: status {status} ({status_name(status)}): {msg}")
        self.status = status


def status_name(s: int) -> str:
    return load().mrw_status_string(s).decode()


def check(status: int, where: str = "mrw") -> None:
    if status != MRW_OK:
        raise MrwError(status, where)


def __getattr__(name):  # mrw.mrw_execute(...) etc. resolve to the raw C entry points
    if name.startswith("mrw_"):
        return getattr(load(), name)
    raise AttributeError(name)


# ------------------------------------------------------------------------------------------------
# Marshalling helpers
# ------------------------------------------------------------------------------------------------
_TORCH_DTYPES = None


def _dtype_code(dt) -> int:
    global _TORCH_DTYPES
    import numpy as np
    if isinstance(dt, np.dtype) or isinstance(dt, type):
        d = np.dtype(dt)
        return {np.dtype(np.uint8): MRW_U8, np.dtype(np.int32): MRW_I32, np.dtype(np.int64): MRW_I64,
                np.dtype(np.float32): MRW_F32, np.dtype(np.float64): MRW_F64, np.dtype(np.complex64): MRW_C64}[d]
    import torch
    if _TORCH_DTYPES is None:
        _TORCH_DTYPES = {torch.uint8: MRW_U8, torch.int32: MRW_I32, torch.int64: MRW_I64, torch.float32: MRW_F32,
                         torch.float64: MRW_F64, torch.bfloat16: MRW_BF16, torch.complex64: MRW_C64}
    return _TORCH_DTYPES[dt]


def buffer(t, epu: int = 0, transfer: int = MRW_PARTITION) -> mrw_buffer:
    """mrw_buffer describing a torch tensor (device or host) or a numpy array (host).

    The last dimension is the row; rows may be padded (the row pitch comes from the stride of
    the second-to-last dimension); outer dimensions must be dense over rows.
    """
    b = mrw_buffer()
    shape = tuple(t.shape)
    if len(shape) < 1 or len(shape) > 4:
        raise ValueError("1..4 dimensions")
    if hasattr(t, "data_ptr"):  # torch
        esz = t.element_size()
        if t.stride(-1) != 1:
            raise ValueError("innermost dimension must be contiguous")
        pitch = t.stride(-2) * esz if t.dim() >= 2 else 0
        b.data = t.data_ptr()
        b.dtype = _dtype_code(t.dtype)
        b.memory = MRW_MEM_DEVICE if t.is_cuda else MRW_MEM_HOST
    else:  # numpy
        esz = t.itemsize
        if t.strides[-1] != esz:
            raise ValueError("innermost dimension must be contiguous")
        pitch = t.strides[-2] if t.ndim >= 2 else 0
        b.data = t.ctypes.data
        b.dtype = _dtype_code(t.dtype)
        b.memory = MRW_MEM_HOST
    b.ndim = len(shape)
    for i, s in enumerate(shape):
        b.shape[i] = int(s)
    b.pitch = int(pitch)
    b.epu = int(epu)
    b.transfer = transfer
    return b


def buffers(*ts) -> ctypes.Array:
    arr = (mrw_buffer * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = t if isinstance(t, mrw_buffer) else buffer(t)
    return arr


def config(fusion=MRW_FUSE_ALL, block=0, ctas_per_sm=0, tile_rows=0, tile_cols=0, unroll=0) -> mrw_config:
    c = mrw_config()
    c.fusion, c.block, c.ctas_per_sm, c.tile_rows, c.tile_cols, c.unroll = fusion, block, ctas_per_sm, tile_rows, \
        tile_cols, unroll
    return c


def params(seed=0, t0=0, t1=0, G=0.0, eps=0.0, dt=0.0, alpha=0.0, nu=0, wg=0) -> mrw_stage_params:
    p = mrw_stage_params()
    p.seed, p.t0, p.t1, p.G, p.eps, p.dt, p.alpha, p.nu, p.wg = seed & 0xFFFFFFFF, t0, t1, G, eps, dt, alpha, nu, wg
    return p


class Node:
    """Owning handle of an mrw_node_t (released on garbage collection)."""

    def __init__(self, handle):
        self.h = ctypes.c_void_p(handle) if not isinstance(handle, ctypes.c_void_p) else handle

    def __del__(self):
        if _lib is not None and self.h:
            _lib.mrw_node_release(self.h)
            self.h = ctypes.c_void_p()


def stage(kind, **kw) -> Node:
    lib = load()
    if isinstance(kind, str):
        kind = STAGE_BY_NAME[kind]
    out = ctypes.c_void_p()
    check(lib.mrw_stage(kind, ctypes.byref(params(**kw)), ctypes.byref(out)), "mrw_stage")
    return Node(out)


def user_stage(name: str, source: str, params=None) -> Node:
    """mrw_stage_user: a u8 stage whose per-pixel device function `name` is defined by the CUDA C
    `source`; `params` are its (at most 8) unsigned 32-bit parameters."""
    vals = [int(v) & 0xFFFFFFFF for v in (params or [])]
    if len(vals) > 8:
        raise ValueError("a user stage takes at most 8 parameters")
    arr = (ctypes.c_uint32 * 8)(*(vals + [0] * (8 - len(vals))))
    out = ctypes.c_void_p()
    check(load().mrw_stage_user(name.encode(), source.encode(), arr, ctypes.byref(out)), "mrw_stage_user")
    return Node(out)


def pipeline(*children) -> Node:
    lib = load()
    out = ctypes.c_void_p()
    check(lib.mrw_pipeline_create(ctypes.byref(out)), "mrw_pipeline_create")
    node = Node(out)
    for c in children:
        check(lib.mrw_pipeline_add_node(node.h, c.h), "mrw_pipeline_add_node")
    return node


def map_(body: Node) -> Node:
    out = ctypes.c_void_p()
    check(load().mrw_map(body.h, ctypes.byref(out)), "mrw_map")
    return Node(out)


def mapreduce(body: Node, op: int = MRW_RED_ADD) -> Node:
    out = ctypes.c_void_p()
    check(load().mrw_mapreduce(body.h, op, ctypes.byref(out)), "mrw_mapreduce")
    return Node(out)


def loop(body: Node, iters: int, kind: int = MRW_LOOP_FOR) -> Node:
    st = mrw_loop_state()
    st.max_iters, st.kind, st.global_sync = iters, kind, 1
    out = ctypes.c_void_p()
    check(load().mrw_loop(body.h, ctypes.byref(st), ctypes.byref(out)), "mrw_loop")
    return Node(out)


def stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Future:
    def __init__(self, h):
        self.h = h

    def wait(self, timeout_ms: int = -1) -> None:
        check(load().mrw_future_wait(self.h, timeout_ms), "mrw_future_wait")

    def result(self, n: int = 3):
        """mrw_future_result: the MapReduce result (n int64 values) as a numpy array."""
        import numpy as np
        out = np.zeros(n, dtype=np.int64)
        check(load().mrw_future_result(self.h, out.ctypes.data, out.nbytes), "mrw_future_result")
        return out

    def elapsed_ms(self) -> float:
        v = ctypes.c_float()
        check(load().mrw_future_elapsed_ms(self.h, ctypes.byref(v)), "mrw_future_elapsed_ms")
        return v.value

    def __del__(self):
        if _lib is not None and self.h:
            _lib.mrw_future_release(self.h)
            self.h = None


def execute(root: Node, args, cfg: mrw_config | None = None, stream=None, timed: bool = False) -> Future:
    """Enqueue root on args (tensors / arrays / mrw_buffer); returns a Future. With timed=True
    the future also records device time (Future.elapsed_ms) through mrw_execute_timed."""
    arr = buffers(*args)
    out = ctypes.c_void_p()
    st = stream_handle(stream) if stream is not None or _cuda_available() else None
    fn = load().mrw_execute_timed if timed else load().mrw_execute
    check(fn(root.h, arr, len(args), ctypes.byref(cfg) if cfg is not None else None, st, ctypes.byref(out)),
          "mrw_execute_timed" if timed else "mrw_execute")
    return Future(out)


def execute_batched(root: Node, in_arena, out_arena, desc, cfg: mrw_config | None = None, stream=None) -> Future:
    import numpy as np
    d = np.ascontiguousarray(desc, dtype=np.int64)
    out = ctypes.c_void_p()
    check(load().mrw_execute_batched(root.h, in_arena.data_ptr(), out_arena.data_ptr(), in_arena.numel(),
                                     d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), d.shape[0],
                                     ctypes.byref(cfg) if cfg is not None else None, stream_handle(stream),
                                     ctypes.byref(out)), "mrw_execute_batched")
    return Future(out)


def fft_schedule_check(nfft: int, nsteps: int, ctas: int) -> dict:
    """Plan and check the L2-ring FFT schedule on the host (mrw_fft_schedule_check)."""
    out = (ctypes.c_int64 * 5)()
    check(load().mrw_fft_schedule_check(nfft, nsteps, ctas, out), "mrw_fft_schedule_check")
    return dict(zip(("slice_rows", "lag_steps", "ring_rows", "ctas", "tickets"), out[:]))


def plan_describe(root: Node, args, cfg: mrw_config | None = None) -> str:
    import json
    arr = buffers(*args)
    need = ctypes.c_int64()
    lib = load()
    check(lib.mrw_plan_describe(root.h, arr, len(args), ctypes.byref(cfg) if cfg else None, None, 0,
                                ctypes.byref(need)), "mrw_plan_describe")
    buf = ctypes.create_string_buffer(need.value)
    check(lib.mrw_plan_describe(root.h, arr, len(args), ctypes.byref(cfg) if cfg else None, buf, need.value,
                                ctypes.byref(need)), "mrw_plan_describe")
    return json.loads(buf.value.decode())


def features(root: Node, args):
    import numpy as np
    f = (ctypes.c_float * MRW_NFEATURES)()
    arr = buffers(*args)
    check(load().mrw_features(root.h, arr, len(args), f), "mrw_features")
    return np.array(f[:], dtype=np.float32)


def tune_candidates(root: Node, args):
    lib = load()
    arr = buffers(*args)
    cnt = ctypes.c_int32()
    check(lib.mrw_tune_candidates(root.h, arr, len(args), None, 0, ctypes.byref(cnt)), "mrw_tune_candidates")
    cfgs = (mrw_config * cnt.value)()
    check(lib.mrw_tune_candidates(root.h, arr, len(args), cfgs, cnt.value, ctypes.byref(cnt)), "mrw_tune_candidates")
    return cfgs


def tune_measure(root: Node, args, cfgs, reps: int = 3, stream=None):
    import numpy as np
    arr = buffers(*args)
    t = (ctypes.c_float * len(cfgs))()
    check(load().mrw_tune_measure(root.h, arr, len(args), cfgs, len(cfgs), reps, stream_handle(stream), t),
          "mrw_tune_measure")
    return np.array(t[:], dtype=np.float64)


def tune(root: Node, args, mode: int = MRW_TUNE_EXHAUSTIVE, reps: int = 3, stream=None):
    arr = buffers(*args)
    best = mrw_config()
    ms = ctypes.c_float()
    check(load().mrw_tune(root.h, arr, len(args), mode, reps, stream_handle(stream), ctypes.byref(best),
                          ctypes.byref(ms)), "mrw_tune")
    return best, ms.value


def _cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


class Model:
    """Owning handle of an mrw_model_t."""

    def __init__(self, k: int, hidden: int = 64, seed: int = 0):
        self.h = ctypes.c_void_p()
        check(load().mrw_model_create(k, hidden, seed, ctypes.byref(self.h)), "mrw_model_create")
        self.k = k
        self.hidden = hidden

    def num_params(self) -> int:
        return load().mrw_model_num_params(self.h)

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        check(load().mrw_model_set_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "mrw_model_set_params")

    def get_params(self):
        import numpy as np
        a = np.zeros(self.num_params(), dtype=np.float32)
        check(load().mrw_model_get_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "mrw_model_get_params")
        return a

    def forward(self, x, y, stream=None):
        check(load().mrw_model_forward(self.h, x.data_ptr(), x.shape[0], y.data_ptr(), stream_handle(stream)),
              "mrw_model_forward")

    def gradients(self, x, t, grads, stream=None) -> float:
        loss = ctypes.c_float()
        check(load().mrw_model_gradients(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], grads.data_ptr(),
                                         ctypes.byref(loss), stream_handle(stream)), "mrw_model_gradients")
        return loss.value

    def adam_step(self, grads, lr: float, stream=None):
        check(load().mrw_model_adam_step(self.h, grads.data_ptr(), lr, stream_handle(stream)), "mrw_model_adam_step")

    def train(self, x, t, epochs: int, batch: int, lr: float, seed: int = 0, stream=None) -> float:
        loss = ctypes.c_float()
        check(load().mrw_model_train(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], epochs, batch, lr, seed,
                                     stream_handle(stream), ctypes.byref(loss)), "mrw_model_train")
        return loss.value

    def install(self, cfgs):
        check(load().mrw_tune_set_model(self.h, cfgs, len(cfgs)), "mrw_tune_set_model")

    def __del__(self):
        if _lib is not None and self.h:
            _lib.mrw_model_release(self.h)
            self.h = ctypes.c_void_p()


def unpack_params(flat, k: int, hidden: int = 64, nin: int = MRW_NFEATURES) -> dict:
    """Split a flat parameter vector into w1, b1, w2, b2, w3, b3 (row-major [out][in])."""
    import numpy as np
    flat = np.asarray(flat)
    sizes = [("w1", (hidden, nin)), ("b1", (hidden,)), ("w2", (hidden, hidden)), ("b2", (hidden,)),
             ("w3", (k, hidden)), ("b3", (k,))]
    out, o = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp)
        o += n
    return out


def pack_params(p: dict):
    import numpy as np
    return np.concatenate([np.asarray(p[k], np.float32).reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


class Balancer:
    """Owning handle of an mrw_balancer_t (CPU + GPU co-execution with dynamic load balancing)."""

    def __init__(self, weight=0.0, max_dev=0.0, c_factor=0.0, trigger=0.0, precision=0.0, gpu_share=-1.0,
                 cpu_threads=0, search_reps=0):
        p = mrw_balance_params()
        p.weight, p.max_dev, p.c_factor, p.trigger, p.precision = weight, max_dev, c_factor, trigger, precision
        p.gpu_share, p.cpu_threads, p.search_reps = gpu_share, cpu_threads, search_reps
        self.h = ctypes.c_void_p()
        check(load().mrw_balancer_create(ctypes.byref(p), ctypes.byref(self.h)), "mrw_balancer_create")

    def observe(self, gpu_ms: float, cpu_ms: float) -> dict:
        r = mrw_balance_report()
        check(load().mrw_balancer_observe(self.h, gpu_ms, cpu_ms, ctypes.byref(r)), "mrw_balancer_observe")
        return r.as_dict()

    def share(self) -> float:
        v = ctypes.c_double()
        check(load().mrw_balancer_share(self.h, ctypes.byref(v)), "mrw_balancer_share")
        return v.value

    def execute(self, root: Node, args, cfg: mrw_config | None = None, stream=None) -> dict:
        """mrw_execute_coexec: blocking; returns the run's balance report."""
        arr = buffers(*args)
        r = mrw_balance_report()
        st = stream_handle(stream) if stream is not None or _cuda_available() else None
        check(load().mrw_execute_coexec(self.h, root.h, arr, len(args), ctypes.byref(cfg) if cfg is not None else None,
                                        st, ctypes.byref(r)), "mrw_execute_coexec")
        return r.as_dict()

    def __del__(self):
        if _lib is not None and self.h:
            _lib.mrw_balancer_release(self.h)
            self.h = ctypes.c_void_p()
