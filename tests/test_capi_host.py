"""Host-side checks of the C ABI that need no GPU: symbols, tree building, validation, plans,
features and the knowledge base. No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import partition
from paper_1510_06585_gb300 import mrw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return mrw.load()


def test_library_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "mrw.h")).read()
    names = set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(mrw_\w+)\s*\(", header, re.M))
    assert len(names) >= 35
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.mrw_abi_version() == 1


def test_status_strings(lib):
    assert lib.mrw_status_string(0) == b"ok"
    assert lib.mrw_status_string(7) == b"timeout"


def _image_args(h=64, w=100, d=None, dtype=np.uint8, reduce=False):
    shape = (h, w) if d is None else (d, h, w)
    a = np.zeros(shape, dtype=dtype)
    b = np.zeros(shape, dtype=np.uint8)
    args = [a, b]
    if reduce:
        args.append(np.zeros(3, np.int64))
    return args


def test_tree_building_and_errors(lib):
    p = mrw.pipeline(mrw.stage("noise", seed=2), mrw.stage("solarise"), mrw.stage("mirror"))
    # a pipeline cannot contain itself
    assert lib.mrw_pipeline_add_node(p.h, p.h) == mrw.MRW_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    assert lib.mrw_stage(99, None, ctypes.byref(out)) == mrw.MRW_ERR_INVALID_ARG
    assert lib.mrw_mapreduce(p.h, 9, ctypes.byref(out)) == mrw.MRW_ERR_INVALID_ARG
    st = mrw.mrw_loop_state()
    st.max_iters = -1
    assert lib.mrw_loop(p.h, ctypes.byref(st), ctypes.byref(out)) == mrw.MRW_ERR_INVALID_ARG
    assert b"max_iters" in lib.mrw_last_error()
    empty = mrw.pipeline()
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(empty, _image_args())
    assert e.value.status == mrw.MRW_ERR_INVALID_ARG


def test_validation_codes_before_any_launch(lib):
    p = mrw.pipeline(mrw.stage("noise", seed=2), mrw.stage("mirror"))
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(p, _image_args(dtype=np.float32))
    assert e.value.status == mrw.MRW_ERR_DTYPE
    a, b = _image_args()
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(p, [a, b[:, :50]])
    assert e.value.status == mrw.MRW_ERR_SHAPE
    # epu must be whole rows
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(p, [mrw.buffer(a, epu=150), b])
    assert e.value.status == mrw.MRW_ERR_CONSTRAINT
    # nu must divide epu (Section 3.1 constraint)
    p2 = mrw.pipeline(mrw.stage("noise", seed=2, nu=7))
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(p2, [mrw.buffer(a, epu=100), b])
    assert e.value.status == mrw.MRW_ERR_CONSTRAINT
    # MapReduce needs the int64 result buffer
    mr = mrw.mapreduce(mrw.map_(mrw.stage("threshold3")))
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(mr, _image_args())
    assert e.value.status == mrw.MRW_ERR_INVALID_ARG
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(mr, _image_args()[:2] + [np.zeros(3, np.int32)])
    assert e.value.status == mrw.MRW_ERR_DTYPE
    # execute refuses bad arguments before touching the GPU
    arr = mrw.buffers(*_image_args(dtype=np.float32))
    fut = ctypes.c_void_p()
    assert lib.mrw_execute(p.h, arr, 2, None, None, ctypes.byref(fut)) == mrw.MRW_ERR_DTYPE
    assert not fut.value
    # a blur inside a Map needs whole planes
    pb = mrw.map_(mrw.stage("blur5"))
    a3, b3 = _image_args(8, 32, d=4)
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(pb, [mrw.buffer(a3, epu=32), b3])
    assert e.value.status == mrw.MRW_ERR_CONSTRAINT
    # unsupported merging function on the device path
    mr_mul = mrw.mapreduce(mrw.stage("threshold3"), mrw.MRW_RED_MUL)
    with pytest.raises(mrw.MrwError) as e:
        mrw.plan_describe(mr_mul, _image_args(reduce=True))
    assert e.value.status == mrw.MRW_ERR_UNSUPPORTED


def test_fused_groups_and_unfused_groups(lib):
    pipe = mrw.pipeline(mrw.stage("noise", seed=1), mrw.stage("solarise"), mrw.stage("mirror"))
    d = mrw.plan_describe(pipe, _image_args(1024, 1024), mrw.config())
    assert d["family"] == "image" and len(d["groups"]) == 1
    g = d["groups"][0]
    assert g["kernel"] == "chain" and g["ops"] == ["noise", "solarise", "mirror"]
    assert g["rows_parallel"] * g["col_vecs"] <= g["grid"] * g["block"]
    u = mrw.plan_describe(pipe, _image_args(1024, 1024), mrw.config(fusion=mrw.MRW_FUSE_NONE))
    assert [x["ops"] for x in u["groups"]] == [["noise"], ["solarise"], ["mirror"]]
    # blur splits prefix / suffix; a second blur opens a new group
    pb = mrw.pipeline(mrw.stage("noise", seed=1), mrw.stage("mirror"), mrw.stage("blur5"), mrw.stage("solarise"),
                      mrw.stage("blur5"))
    d = mrw.plan_describe(pb, _image_args(300, 333))
    # a group with pointwise stages after its blur runs on the 2-D tile kernel; a blur with only a
    # prefix on the row-streaming kernel, whose work items are strips of 124 columns
    assert [x["kernel"] for x in d["groups"]] == ["stencil", "stencil_rows"]
    assert d["groups"][0]["pre"] == ["noise", "mirror"] and d["groups"][0]["suf"] == ["solarise"]
    assert d["groups"][1]["pre"] == [] and d["groups"][1]["blur"]
    # stencil tiles cover the plane
    g0 = d["groups"][0]
    assert g0["tiles_x"] * g0["tile"][1] >= 333 and (g0["tiles_x"] - 1) * g0["tile"][1] < 333
    assert g0["tiles_y"] * g0["tile"][0] >= 300 and (g0["tiles_y"] - 1) * g0["tile"][0] < 300
    g1 = d["groups"][1]
    assert g1["tile"][1] == 124 and g1["tiles_x"] == 3 and g1["tiles_y"] * g1["tile"][0] >= 300
    # three noise stages do not fit one chain group's registers
    p3 = mrw.pipeline(*[mrw.stage("noise", seed=s) for s in range(3)])
    assert len(mrw.plan_describe(p3, _image_args())["groups"]) == 2


def test_mapreduce_fuses_into_the_last_chain_group(lib):
    mr = mrw.mapreduce(mrw.map_(mrw.stage("threshold3")))
    args = _image_args(64, 512, d=8, reduce=True)
    d = mrw.plan_describe(mr, args, mrw.config())
    assert len(d["groups"]) == 1 and d["groups"][0]["reduce"] == 1
    assert d["groups"][0]["finish_kernel"]  # the one-CTA finish runs behind the reducing launch
    u = mrw.plan_describe(mr, args, mrw.config(fusion=mrw.MRW_FUSE_NONE))
    assert len(u["groups"]) == 2 and u["groups"][1]["reduce_only"]
    assert [g["finish_kernel"] for g in u["groups"]] == [False, True]
    # a reducing group's CTAs do not wait at their end, so it takes the map's launch shape
    cfg = mrw.config(block=128, ctas_per_sm=8, unroll=8)
    big = _image_args(512, 512, d=512, reduce=True)
    g_red = mrw.plan_describe(mr, big, cfg)["groups"][0]
    g_map = mrw.plan_describe(mrw.map_(mrw.stage("threshold3")), big[:2], cfg)["groups"][0]
    assert (g_red["grid"], g_red["block"], g_red["rows_parallel"]) == (g_map["grid"], g_map["block"],
                                                                       g_map["rows_parallel"])
    assert g_red["grid"] * g_red["block"] == g_red["rows_parallel"] * g_red["col_vecs"] and g_red["order"] == "blocked"
    # pageable host buffers of 8 MiB and more are staged in overlapped chunks whose kernels add into
    # the zeroed result: no finish kernel; below that size the whole image is staged and finished
    assert d["staging"] == "whole"
    chunked = mrw.plan_describe(mr, big, cfg)
    assert chunked["staging"] == "chunked" and chunked["groups"][0]["finish_kernel"] is False


def test_loops_of_image_stages_unroll_into_the_chain(lib):
    body = mrw.pipeline(mrw.stage("solarise"), mrw.stage("mirror"))
    d = mrw.plan_describe(mrw.loop(body, 3), _image_args())
    assert d["groups"][0]["ops"] == ["solarise", "mirror"] * 3


def _nbody_args(n):
    return [np.zeros((n, 4), np.float32) for _ in range(3)]


def test_nbody_plan_partitions_satisfy_constraints(lib):
    kdk = mrw.stage("nbody_kdk", eps=1e-3, dt=1e-3)
    tree = mrw.pipeline(mrw.stage("nbody_accel", eps=1e-3, dt=1e-3), mrw.loop(kdk, 100))
    for n in (1, 7, 1000, 65536, 100003):
        for cfg in (mrw.config(), mrw.config(ctas_per_sm=4, tile_rows=4), mrw.config(tile_rows=1)):
            d = mrw.plan_describe(tree, _nbody_args(n), cfg)
            assert [s["kind"] for s in d["steps"]] == ["accel", "kdk"]
            assert d["steps"][1]["iters"] == 100 and d["steps"][1]["loop"] == "device_graph"
            parts = [tuple(p) for p in d["partitions"]]
            assert partition.check_plan(n, [p for p in parts if p[1] > 0], epu=1, nu=1) == []
            # each CTA's partition fits its threads
            assert max(p[1] for p in parts) <= d["threads_per_group"] * d["bodies_per_thread"]
            assert d["block"] == 4 * d["threads_per_group"] and d["threads_per_group"] % 32 == 0
    u = mrw.plan_describe(tree, _nbody_args(64), mrw.config(fusion=mrw.MRW_FUSE_NONE))
    assert u["steps"][1]["loop"] == "host"
    with pytest.raises(mrw.MrwError):
        mrw.plan_describe(mrw.stage("nbody_kdk", eps=0.0, dt=1e-3), _nbody_args(8))


def test_features_describe_the_tree(lib):
    p = mrw.pipeline(mrw.stage("noise", seed=1), mrw.stage("noise", seed=2), mrw.stage("mirror"),
                     mrw.stage("blur5"))
    f = mrw.features(p, _image_args(256, 1000))
    assert f.shape == (16,)
    assert f[0] == 1 and f[1] == 0 and f[2] == 0 and f[3] == 0
    assert f[4] == 4 and f[5] == 2 and f[7] == 1 and f[8] == 1
    assert abs(f[9] - np.log2(256 * 1000)) < 1e-5 and f[12] == 1
    mr = mrw.mapreduce(mrw.stage("threshold3"))
    assert mrw.features(mr, _image_args(64, 64, reduce=True))[3] == 1


def test_knowledge_base_roundtrip(lib, tmp_path):
    path = tmp_path / "kb.txt"
    path.write_text("P(S1{0,0,0,0x0p+0,0x0p+0,0x0p+0,0x0p+0,0,0})|0:2:8x8x;\t1 128 4 16 64 2\t0.5\t0\n")
    assert lib.mrw_kb_clear() == 0
    assert lib.mrw_kb_load(str(path).encode()) == 0
    assert lib.mrw_kb_size() == 1
    out = tmp_path / "kb2.txt"
    assert lib.mrw_kb_save(str(out).encode()) == 0
    assert out.read_text() == path.read_text()
    bad = tmp_path / "bad.txt"
    for text in ("only-one-field\n", "k\t1 128 4 16 64 2\tfast\t0\n", "k\t1 128 4 16 64 2\t0.5\t1x\n",
                 "k\t1 128 4 16 64 2\t\t0\n", "k\t1 128 4 16 64 2\t0.5\t99999999999\n", "k\t1 128\t0.5\t0\n"):
        bad.write_text(text)
        assert lib.mrw_kb_load(str(bad).encode()) == mrw.MRW_ERR_INVALID_ARG, text
    assert lib.mrw_kb_size() == 1  # a failed load adds nothing
    crlf = tmp_path / "crlf.txt"
    crlf.write_text(path.read_text().replace("\n", "\r\n"))
    assert lib.mrw_kb_clear() == 0 and lib.mrw_kb_load(str(crlf).encode()) == 0 and lib.mrw_kb_size() == 1
    lib.mrw_kb_clear()


def test_candidates_are_sixteen_valid_configs(lib):
    p = mrw.pipeline(mrw.stage("noise", seed=1))
    cfgs = mrw.tune_candidates(p, _image_args())
    assert len(cfgs) == 16
    assert cfgs[0].fusion == mrw.MRW_FUSE_ALL and cfgs[8].fusion == mrw.MRW_FUSE_NONE
    assert len({c.as_tuple() for c in cfgs}) == 16


def test_while_changed_loops_are_planned_and_validated(lib):
    blur = mrw.stage("blur5")
    w = mrw.loop(blur, 500, mrw.MRW_LOOP_WHILE_CHANGED)
    d = mrw.plan_describe(mrw.pipeline(mrw.stage("noise", seed=1), w, mrw.stage("solarise")), _image_args(40, 50))
    assert d["while_changed"] == {"first_stage": 1, "end_stage": 2, "max_iters": 500, "body_kernels": 1}
    with pytest.raises(mrw.MrwError) as e:   # one convergence loop per tree
        mrw.plan_describe(mrw.pipeline(w, mrw.loop(blur, 3, mrw.MRW_LOOP_WHILE_CHANGED)), _image_args())
    assert e.value.status == mrw.MRW_ERR_UNSUPPORTED
    with pytest.raises(mrw.MrwError) as e:   # not inside a MapReduce
        mrw.plan_describe(mrw.mapreduce(mrw.pipeline(w, mrw.stage("threshold3"))), _image_args(reduce=True))
    assert e.value.status == mrw.MRW_ERR_UNSUPPORTED
    with pytest.raises(mrw.MrwError) as e:   # image trees only
        mrw.plan_describe(mrw.loop(mrw.stage("nbody_kdk", eps=1e-3, dt=1e-3), 5, mrw.MRW_LOOP_WHILE_CHANGED),
                          _nbody_args(16))
    assert e.value.status == mrw.MRW_ERR_UNSUPPORTED


@pytest.mark.parametrize("names, pattern", [
    (["noise", "solarise", "mirror"], "noise_solarise"),
    (["mirror", "noise", "mirror", "solarise"], "noise_solarise"),
    (["solarise", "noise"], "generic"),
    (["noise", "noise"], "generic"),
    (["noise", "solarise", "solarise"], "generic"),
    (["noise"], "noise"),
    (["mirror", "solarise"], "solarise"),
    (["mirror"], "none"),
    (["mirror", "mirror"], "none"),
    (["threshold3", "mirror"], "threshold3"),
    (["solarise", "threshold3"], "generic"),
])
def test_op_sequences_the_kernels_run_without_interpretation(lib, names, pattern):
    """The host classifies each fused group's op list; mirrors move no data and do not count."""
    pipe = mrw.pipeline(*[mrw.stage(n, seed=3) if n == "noise" else mrw.stage(n) for n in names])
    g = mrw.plan_describe(pipe, _image_args(64, 256))["groups"]
    assert len(g) == 1 and g[0]["kernel"] == "chain" and g[0]["pattern"] == pattern
    u = mrw.plan_describe(pipe, _image_args(64, 256), mrw.config(fusion=mrw.MRW_FUSE_NONE))["groups"]
    single = {"noise": "noise", "solarise": "solarise", "mirror": "none", "threshold3": "threshold3"}
    assert [x["pattern"] for x in u] == [single[n] for n in names]


def test_blur_prefix_sequences(lib):
    d = mrw.plan_describe(mrw.pipeline(mrw.stage("noise", seed=2), mrw.stage("solarise"), mrw.stage("mirror"),
                                       mrw.stage("blur5")), _image_args(300, 333))["groups"]
    assert [x["kernel"] for x in d] == ["stencil_rows"] and d[0]["pre_pattern"] == "noise_solarise"
    d = mrw.plan_describe(mrw.pipeline(mrw.stage("blur5")), _image_args(300, 333))["groups"]
    assert d[0]["pre_pattern"] == "none"
    d = mrw.plan_describe(mrw.pipeline(mrw.stage("solarise"), mrw.stage("noise", seed=1), mrw.stage("blur5"),
                                       mrw.stage("solarise")), _image_args(300, 333))["groups"]
    assert d[0]["kernel"] == "stencil" and d[0]["pre_pattern"] == "generic"


def test_future_result_rejects_null_arguments(lib):
    out = np.zeros(3, dtype=np.int64)
    assert lib.mrw_future_result(None, out.ctypes.data, out.nbytes) == mrw.MRW_ERR_INVALID_ARG


def test_saxpy_stages_fuse_into_passes_of_64(lib):
    x = np.zeros(1000, np.float32)
    y = np.zeros(1000, np.float32)
    tree = mrw.loop(mrw.stage("saxpy", alpha=0.5), 100)
    d = mrw.plan_describe(tree, [x, y])
    assert d["family"] == "saxpy" and d["stages"] == 100 and d["launches"] == 2 and d["n"] == 1000
    assert mrw.plan_describe(tree, [x, y], mrw.config(fusion=mrw.MRW_FUSE_NONE))["launches"] == 100
    assert mrw.plan_describe(tree, [x, y], mrw.config(unroll=8))["grid"] == 1


def test_batched_descriptor_offsets_near_int64_max_are_rejected_before_any_launch(lib):
    # validation runs before anything touches the GPU or the arenas (the pointers are never used)
    tree = mrw.map_(mrw.pipeline(mrw.stage("noise"), mrw.stage("blur5")))
    desc = np.array([[0, 8, 8, 16, 1], [(1 << 63) - 16, 8, 8, 16, 2]], dtype=np.int64)
    dptr = desc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    fut = ctypes.c_void_p()
    a, b = 1 << 20, 1 << 21  # two non-overlapping 16-byte aligned addresses, 4096 bytes each
    assert lib.mrw_execute_batched(tree.h, a, b, 4096, dptr, 2, None, None, ctypes.byref(fut)) == mrw.MRW_ERR_SHAPE
    assert lib.mrw_execute_batched_noalloc(tree.h, a, b, 4096, dptr, 2, None, None) == mrw.MRW_ERR_SHAPE
    assert b"outside the arena" in lib.mrw_last_error()


def test_empty_buffers_are_refused_before_any_launch(lib):
    fut = ctypes.c_void_p()
    cases = [
        (mrw.pipeline(mrw.stage("noise", seed=1)), [np.zeros((0, 16), np.uint8), np.zeros((0, 16), np.uint8)]),
        (mrw.mapreduce(mrw.map_(mrw.stage("threshold3"))),
         [np.zeros((4, 0, 16), np.uint8), np.zeros((4, 0, 16), np.uint8), np.zeros(3, np.int64)]),
        (mrw.map_(mrw.stage("saxpy", alpha=2.0)), [np.zeros(0, np.float32), np.zeros(0, np.float32)]),
        (mrw.stage("nbody_accel", eps=1e-3), [np.zeros((0, 4), np.float32)] * 3),
        (mrw.pipeline(mrw.stage("fft")), [np.zeros((0, 65536), np.complex64)] * 2),
    ]
    keep = []
    for tree, args in cases:
        arr = (mrw.mrw_buffer * len(args))()
        for i, a in enumerate(args):  # described by hand: numpy gives empty arrays arbitrary strides
            b = np.zeros(16, np.uint8)
            keep.append(b)
            arr[i].data = b.ctypes.data
            arr[i].dtype = mrw._dtype_code(a.dtype)
            arr[i].ndim = a.ndim
            for d, e in enumerate(a.shape):
                arr[i].shape[d] = e
            arr[i].memory = mrw.MRW_MEM_HOST
        assert lib.mrw_execute(tree.h, arr, len(args), None, None, ctypes.byref(fut)) == mrw.MRW_ERR_SHAPE
        assert not fut.value


def test_fft_ring_schedule_gives_every_item_one_ticket_and_waits_only_backwards(lib):
    # the persistent FFT grid claims work items in ticket order and waits only for smaller tickets
    # (checked exhaustively on the host for every plan here); phase p + 1 of a row trails phase p
    # by about 2.5 grids of tickets, and the ring holds at most (P - 1) L + 3 slices of rows
    for ctas in (1, 7, 152, 456):
        for nsteps in (1, 2, 3, 8):
            for nfft in (1, 2, 5, 36, 37, 83, 256, 1000):
                r = mrw.fft_schedule_check(nfft, nsteps, ctas)
                P, G, L = nsteps + 1, r["slice_rows"], r["lag_steps"]
                slices = -(-nfft // G)
                assert r["tickets"] == slices * G * 16 * P and r["ctas"] == min(ctas, r["tickets"])
                assert 1 <= L <= 2 and (L == 2 or slices < 2)
                assert r["ring_rows"] == min(slices, (P - 1) * L + 3) * G
                if slices >= 2:
                    assert 16 * G * L * P >= 2.5 * ctas  # the lag between a row's phases, in tickets
    with pytest.raises(mrw.MrwError) as e:
        mrw.fft_schedule_check(0, 2, 152)
    assert e.value.status == mrw.MRW_ERR_UNSUPPORTED
    with pytest.raises(mrw.MrwError) as e:
        mrw.fft_schedule_check(4, 9, 152)
    assert e.value.status == mrw.MRW_ERR_UNSUPPORTED
