"""Host logic of CPU + GPU co-execution (Section 3.3 of the paper): the load balancing threshold
lbt, the binary search of the workload distribution generator (Section 3.2) and the adaptive
binary search, driven through mrw_balancer_observe with synthetic times; no GPU needed."""
import numpy as np
import pytest

from paper_1510_06585_gb300 import mrw as M


@pytest.fixture(scope="module", autouse=True)
def lib():
    return M.load()


def _linear(share, rate_gpu, rate_cpu, work=1000.0):
    """Times of the two shares when each side processes its rows at a fixed rate."""
    return share * work / rate_gpu, (1.0 - share) * work / rate_cpu


def test_lbt_of_consecutive_unbalanced_runs_is_one_minus_a_third_to_the_n():
    b = M.Balancer(gpu_share=0.5)  # monitoring a converged profile
    for n in range(1, 4):
        r = b.observe(1.0, 10.0)  # dev = 0.1 < 0.85: unbalanced
        assert r["unbalanced"] == 1 and r["dev"] == pytest.approx(0.1)
        assert r["lbt"] == pytest.approx(1.0 - (1.0 / 3.0) ** n)
    # three consecutive unbalanced runs from lbt = 0 reach 26/27 >= 0.95: the load balancer started
    assert r["phase"] == M.MRW_BAL_SHIFT


def test_balanced_runs_keep_lbt_down_and_history_decays():
    b = M.Balancer(gpu_share=0.5)
    r = b.observe(1.0, 1.1)  # dev = 0.909 >= 0.85: balanced
    assert r["unbalanced"] == 0 and r["lbt"] == 0.0 and r["phase"] == M.MRW_BAL_MONITOR
    assert b.observe(1.0, 2.0)["lbt"] == pytest.approx(2.0 / 3.0)
    r = b.observe(1.0, 1.0)
    assert r["lbt"] == pytest.approx(2.0 / 9.0)  # the unbalanced run weighs (1 - 2/3) one run later
    assert r["next_share"] == 0.5  # no persistent imbalance: nothing moves


def test_c_factor_and_max_dev_set_the_threshold():
    b = M.Balancer(gpu_share=0.5, max_dev=0.8, c_factor=0.9)
    assert b.observe(0.73, 1.0)["unbalanced"] == 0  # 0.73 / 0.9 = 0.811 >= 0.8
    assert b.observe(0.71, 1.0)["unbalanced"] == 1  # 0.71 / 0.9 = 0.789 < 0.8


def test_profile_construction_is_a_binary_search():
    b = M.Balancer(precision=1.0 / 64)
    shares, sizes = [], []
    for _ in range(6):  # the GPU always faster: it keeps the half it was offered each time
        r = b.observe(1.0, 2.0)
        shares.append(r["gpu_share"])
        sizes.append(r["transferable"])
    assert shares == [1.0 - 2.0 ** -(n + 1) for n in range(6)]
    assert sizes == [2.0 ** -(n + 1) for n in range(6)]  # transferableSize(n) = size / 2^n
    assert r["phase"] == M.MRW_BAL_SEARCH  # 1/64 is not below the precision yet
    assert b.observe(1.0, 2.0)["phase"] == M.MRW_BAL_MONITOR  # 1/128 is: the profile is built
    c = M.Balancer(precision=1.0 / 8)
    assert [c.observe(3.0, 1.0)["gpu_share"] for _ in range(3)] == [0.5, 0.25, 0.125]


@pytest.mark.parametrize("rate_gpu,rate_cpu", [(3.0, 1.0), (1.0, 1.0), (10.0, 1.0), (1.0, 4.0)])
def test_search_converges_to_the_balance_point(rate_gpu, rate_cpu):
    b = M.Balancer(precision=1.0 / 256)
    for _ in range(20):
        r = b.observe(*_linear(b.share(), rate_gpu, rate_cpu))
        if r["phase"] == M.MRW_BAL_MONITOR:
            break
    want = rate_gpu / (rate_gpu + rate_cpu)
    assert abs(b.share() - want) <= 1.0 / 256
    tg, tc = _linear(b.share(), rate_gpu, rate_cpu)
    assert min(tg, tc) / max(tg, tc) >= 0.95


def test_adaptive_search_shifts_doubles_then_bisects_after_a_load_change():
    # converged at 0.75 for GPU : CPU rates 3 : 1; then the host cores slow down 3x (rates 3 : 1/3,
    # balance point 0.9)
    b = M.Balancer(gpu_share=0.75, precision=1.0 / 256)
    assert b.observe(*_linear(0.75, 3.0, 1.0))["unbalanced"] == 0
    trace = []
    for _ in range(40):
        s = b.share()
        r = b.observe(*_linear(s, 3.0, 1.0 / 3.0))
        trace.append((s, r["phase"], r["transferable"]))
        if r["phase"] == M.MRW_BAL_MONITOR and len(trace) > 3:
            break
    shares = [t[0] for t in trace]
    # three unbalanced runs at 0.75 (lbt 2/3, 8/9, 26/27), then shifts of 1/16, 1/16 and a doubled 1/8
    assert shares[:3] == [0.75, 0.75, 0.75]
    assert shares[3] == pytest.approx(0.75 + 1 / 16) and shares[4] == pytest.approx(0.75 + 2 / 16)
    assert trace[4][1] == M.MRW_BAL_SHIFT and trace[4][2] == pytest.approx(1 / 8)
    assert any(t[1] == M.MRW_BAL_BISECT for t in trace)
    assert abs(b.share() - 0.9) <= 1.0 / 128
    assert len(trace) <= 16


def test_balancer_parameter_errors():
    lib = M.load()
    import ctypes
    out = ctypes.c_void_p()
    for bad in ({"weight": 1.5}, {"max_dev": -0.1}, {"precision": 2.0}, {"c_factor": -1.0}, {"gpu_share": 1.5},
                {"cpu_threads": -1}, {"search_reps": -1}, {"search_reps": 65}):
        p = M.mrw_balance_params()
        for k, v in bad.items():
            setattr(p, k, v)
        assert lib.mrw_balancer_create(ctypes.byref(p), ctypes.byref(out)) == M.MRW_ERR_INVALID_ARG, bad
    b = M.Balancer()
    assert lib.mrw_balancer_observe(b.h, -1.0, 1.0, None) == M.MRW_ERR_INVALID_ARG
    assert lib.mrw_balancer_observe(b.h, float("nan"), 1.0, None) == M.MRW_ERR_INVALID_ARG
    assert lib.mrw_execute_coexec(None, None, None, 0, None, None, None) == M.MRW_ERR_INVALID_ARG


def test_search_reps_take_the_fastest_time_of_each_side():
    b = M.Balancer(search_reps=2, precision=1.0 / 4)
    # at share 0.5 a slow first GPU run (a cold start) does not decide: the second, faster one does
    r = b.observe(9.0, 2.0)
    assert r["next_share"] == 0.5 and r["phase"] == M.MRW_BAL_SEARCH
    r = b.observe(1.0, 2.0)
    assert r["next_share"] == 0.75  # the GPU was faster at its best: it keeps its half
