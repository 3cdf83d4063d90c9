"""GPU parity of the FFT stages (Section 4, FFT pipelined with its inversion) against the FP64
oracle: rows of 65,536 complex float32 values, one cluster of 8 or 16 CTAs per row, or work items
of a persistent grid exchanging through an L2-resident ring.

Tolerance: normwise relative error per row <= 1e-5. A float32 transform of 2^16 points goes
through 16 radix-2-equivalent levels, each adding a rounding error of a few units of 2^-24 to the
row's norm, plus one rounded twiddle per value per level group: about 1e-6 in the worst row; a
wrong twiddle, sign or index anywhere gives an error of order 1."""
import numpy as np
import pytest
import torch

from oracle import fft as F
from paper_1510_06585_gb300 import inputs
from paper_1510_06585_gb300 import mrw as M

pytestmark = pytest.mark.gpu
N = 65536
TOL = 1e-5


def tree_of(names):
    return M.pipeline(*[M.stage(n) for n in names])


def run(tree, x, cfg=None, inplace=False, host=False):
    if host:
        xd = torch.from_numpy(x.copy())
        yd = xd if inplace else torch.empty_like(xd)
    else:
        xd = torch.from_numpy(x).cuda()
        yd = xd if inplace else torch.empty_like(xd)
    M.execute(tree, [xd, yd], cfg).wait(120000)
    return yd.cpu().numpy()


@pytest.mark.parametrize("names", [["fft"], ["ifft"], ["fft", "ifft"], ["ifft", "fft"], ["fft", "fft"]])
def test_pipelines_match_the_oracle_fused_and_per_stage(names):
    x = inputs.fft_signals(5, N, seed=len(names) * 7 + (names[0] == "fft"))
    want = F.pipeline(x, names)
    for cfg in (M.config(), M.config(fusion=M.MRW_FUSE_NONE)):
        got = run(tree_of(names), x, cfg)
        assert F.rel_error(got, want) <= TOL, (names, cfg.fusion, F.rel_error(got, want))


@pytest.mark.parametrize("cps", [0, 1])  # the default (a cluster per row at 3 rows) and the L2-ring form
def test_closed_forms(cps):
    x = np.zeros((3, N), np.complex64)
    x[0, 0] = 1.0                                              # impulse -> all ones
    k0 = 4321
    x[1] = np.exp(2j * np.pi * k0 * np.arange(N) / N)          # exponential -> N at k0
    x[2] = 0.75 - 0.25j                                        # constant -> N (0.75 - 0.25i) at 0
    X = run(tree_of(["fft"]), x, M.config(ctas_per_sm=cps)).astype(np.complex128)
    assert np.abs(X[0] - 1.0).max() <= 1e-6
    assert abs(X[1, k0] - N) <= 1e-3 * N ** 0.5 and np.abs(np.delete(X[1], k0)).max() <= 1e-3 * N ** 0.5
    assert abs(X[2, 0] - N * (0.75 - 0.25j)) <= 1e-3 and np.abs(X[2, 1:]).max() <= 1e-3
    # the inverse of the impulse's transform is the impulse: N^-1 sum_k e^(+2 pi i k n / N) = [n = 0]
    y = run(tree_of(["ifft"]), X[:1].astype(np.complex64), M.config(ctas_per_sm=cps)).astype(np.complex128)
    assert abs(y[0, 0] - 1.0) <= 1e-6 and np.abs(y[0, 1:]).max() <= 1e-6


def test_forward_then_inverse_returns_the_input_and_matches_per_stage():
    x = inputs.fft_signals(7, N, seed=11)
    tree = tree_of(["fft", "ifft"])
    fused = run(tree, x)
    per_stage = run(tree, x, M.config(fusion=M.MRW_FUSE_NONE))
    assert F.rel_error(fused, x) <= TOL and F.rel_error(per_stage, x) <= TOL
    assert F.rel_error(fused, per_stage) <= 2 * TOL


def test_long_chains_more_rows_than_clusters_in_place_and_host_buffers():
    # 10 alternating transforms need two fused launches (8 + 2); 83 rows are more than the
    # clusters resident at once and not a multiple of their number
    x = inputs.fft_signals(83, N, seed=5)
    loop = M.loop(tree_of(["fft", "ifft"]), 5)
    got = run(loop, x)
    assert F.rel_error(got, x) <= 4 * TOL
    want = F.fft_rows(x)
    assert F.rel_error(run(tree_of(["fft"]), x, inplace=True), want) <= TOL
    assert F.rel_error(run(tree_of(["fft"]), x[:3], host=True), want[:3]) <= TOL
    assert F.rel_error(run(tree_of(["fft"]), x[:2], host=True, inplace=True), want[:2]) <= TOL
    ring = M.config(ctas_per_sm=1)  # the L2-ring form on host buffers, out of place and in place
    assert F.rel_error(run(tree_of(["fft"]), x[:41], ring, host=True), want[:41]) <= TOL
    assert F.rel_error(run(tree_of(["ifft", "fft"]), x[:7], ring, host=True, inplace=True), x[:7]) <= TOL


def test_one_row_and_plan():
    x = inputs.fft_signals(1, N, seed=2)[0]  # a 1-D buffer is one row
    assert F.rel_error(run(tree_of(["ifft"]), x), F.ifft_rows(x)) <= TOL
    d = M.plan_describe(M.loop(M.stage("fft"), 9), [torch.from_numpy(inputs.fft_signals(2, N)).cuda()] * 2)
    assert d["family"] == "fft" and [len(l) for l in d["launches"]] == [8, 1] and d["cluster"] in (4, 8, 16)


def test_rejects_bad_shapes_and_types():
    bad = torch.zeros(2, 4096, dtype=torch.complex64, device="cuda")
    with pytest.raises(M.MrwError) as e:
        M.execute(tree_of(["fft"]), [bad, bad])
    assert e.value.status == M.MRW_ERR_SHAPE
    f32 = torch.zeros(2, N, dtype=torch.float32, device="cuda")
    with pytest.raises(M.MrwError) as e:
        M.execute(tree_of(["fft"]), [f32, f32])
    assert e.value.status == M.MRW_ERR_DTYPE
    with pytest.raises(M.MrwError) as e:
        M.execute(M.pipeline(M.stage("fft"), M.stage("solarise")), [bad, bad])
    assert e.value.status == M.MRW_ERR_UNSUPPORTED


def test_full_size_256_rows_128_mb():
    x = inputs.fft_signals(256, N)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    M.execute(tree_of(["fft", "ifft"]), [xd, yd]).wait(120000)
    assert F.rel_error(yd.cpu().numpy(), x) <= TOL
    M.execute(tree_of(["fft"]), [xd, yd]).wait(120000)
    rows = [0, 37, 128, 255]
    assert F.rel_error(yd.cpu().numpy()[rows], F.fft_rows(x[rows])) <= TOL


def test_tmem_form_runs_more_clusters_at_once():
    # the form that parks the exchange's values in tensor memory exists to fit three CTAs per SM
    x = torch.zeros(2, N, dtype=torch.complex64, device="cuda")
    reg = M.plan_describe(tree_of(["fft"]), [x, x], M.config(ctas_per_sm=2))
    tm = M.plan_describe(tree_of(["fft"]), [x, x], M.config(ctas_per_sm=4))
    assert not reg["tmem"] and tm["tmem"] and tm["clusters_resident"] > reg["clusters_resident"] > 0


@pytest.mark.parametrize("cps,form", [(0, None), (1, "l2"), (2, "reg"), (3, "c16"), (4, "tmem")])
def test_every_kernel_form_on_every_row_count(cps, form):
    # clusters of 8 CTAs with the exchange's values in registers (two CTAs per SM) or in tensor
    # memory (three per SM), clusters of 16 CTAs (bulk copies between the CTAs' shared memory), and
    # the persistent grid of work items over an L2-resident ring (the default once the rows
    # outnumber the register form's resident clusters, form None here), chosen by the
    # configuration, on row counts below, at and above the number of clusters that run at once, in
    # place and out of place, and through a 3-transform fused launch
    cfg = M.config(ctas_per_sm=cps)
    for nfft in (1, 5, 23, 40, 61):
        x = inputs.fft_signals(nfft, N, seed=nfft)
        xs = [torch.from_numpy(x).cuda()] * 2
        d = M.plan_describe(tree_of(["fft"]), xs, cfg)
        want = form if form is not None else \
            ("l2" if nfft > M.plan_describe(tree_of(["fft"]), xs, M.config(ctas_per_sm=2))["clusters_resident"] else "reg")
        assert d["form"] == want, (nfft, d)
        if want == "l2":
            assert d["schedule_ok"] and d["ctas"] > 0 and d["ring_rows"] >= d["slice_rows"]
        else:
            assert d["cluster"] == (16 if want == "c16" else 8) and d["tmem"] == (want == "tmem")
            assert d["clusters_resident"] > 0
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        M.execute(tree_of(["fft", "ifft", "fft"]), [xd, yd], cfg).wait(60000)
        assert F.rel_error(yd.cpu().numpy(), F.pipeline(x, ["fft", "ifft", "fft"])) <= TOL, nfft
        M.execute(tree_of(["ifft"]), [xd, xd], cfg).wait(60000)
        assert F.rel_error(xd.cpu().numpy(), F.ifft_rows(x)) <= TOL, nfft


def test_ring_form_wait_gives_up_and_reports_without_hanging():
    # A child process runs the L2-ring form with its dependency waits told to give up at once:
    # items claimed before the items they read have finished give up, the kernel records it in the
    # status word and runs out its tickets, the future reports it, and the stream stays usable.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r"""
import os, sys, torch
sys.path.insert(0, %r)
from paper_1510_06585_gb300 import mrw as M, inputs
from oracle import fft as F
x = inputs.fft_signals(2, 65536, seed=3)
xd = torch.from_numpy(x).cuda(); yd = torch.empty_like(xd)
t = M.pipeline(M.stage("fft"), M.stage("ifft"))
f = M.execute(t, [xd, yd], M.config(ctas_per_sm=1))
print("status", M.load().mrw_future_wait(f.h, 60000))
os.environ.pop("MRW_TEST_WAIT_POLLS")
M.execute(t, [xd, yd], M.config(ctas_per_sm=1)).wait(60000)
print("after", F.rel_error(yd.cpu().numpy(), x) <= 1e-5)
""" % root
    env = dict(os.environ, MRW_TEST_WAIT_POLLS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "status %d" % M.MRW_ERR_DEVICE in r.stdout, r.stdout
    assert "after True" in r.stdout, r.stdout


def test_ring_form_reuses_its_slots_many_times():
    # 700 rows: about six times the ring's rows, so most rows wait for the row that last held their
    # slot; every row of the pair comes back to its input, and sampled rows of a single transform
    # match the oracle
    x = inputs.fft_signals(700, N, seed=17)
    ring = M.config(ctas_per_sm=1)
    d = M.plan_describe(tree_of(["fft", "ifft"]), [torch.zeros(700, N, dtype=torch.complex64, device="cuda")] * 2, ring)
    assert d["form"] == "l2" and d["schedule_ok"] and 700 >= 5 * d["ring_rows"], d
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    M.execute(tree_of(["fft", "ifft"]), [xd, yd], ring).wait(120000)
    y = yd.cpu().numpy()
    assert max(F.rel_error(y[i:i + 100], x[i:i + 100]) for i in range(0, 700, 100)) <= TOL
    M.execute(tree_of(["fft"]), [xd, yd], ring).wait(120000)
    rows = [0, 111, 112, 350, 699]
    assert F.rel_error(yd.cpu().numpy()[rows], F.fft_rows(x[rows])) <= TOL
