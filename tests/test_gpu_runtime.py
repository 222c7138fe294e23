"""Runtime behaviour of the library on the GPU: replaying the captured step
graphs gives the same bits as launching the kernels one by one, the two mixed
launches per step give the same bits as separate L.eta / predictor /
corrector launches, profiling records every launch, sharded trajectory
offsets reproduce the unsharded run."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(prec, steps, graph, N=200, M=70, offset=0, traj=None):
    from paper_2608_10075_b300 import twa
    old = os.environ.pop("TWA_NO_GRAPH", None)
    if not graph:
        os.environ["TWA_NO_GRAPH"] = "1"
    try:
        with twa.TWA(N, 1.0, 20.0, 1.0, 1e-3, seed=4, precision=prec, traj_offset=offset) as g:
            g.run(M, steps)
            return g.get_state()
    finally:
        os.environ.pop("TWA_NO_GRAPH", None)
        if old is not None:
            os.environ["TWA_NO_GRAPH"] = old


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("N,M,steps", [(200, 70, 9), (300, 130, 6), (37, 5, 5)])
def test_mixed_launches_equal_separate_launches(prec, N, M, steps):
    # L.eta tiles of step t + 1 inside the launches of step t, scheduled by the
    # host, versus a launch of their own at the start of each step
    old = os.environ.pop("TWA_SEPARATE_LETA", None)
    try:
        a = _run(prec, steps, graph=True, N=N, M=M)
        os.environ["TWA_SEPARATE_LETA"] = "1"
        b = _run(prec, steps, graph=True, N=N, M=M)
    finally:
        os.environ.pop("TWA_SEPARATE_LETA", None)
        if old is not None:
            os.environ["TWA_SEPARATE_LETA"] = old
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_graph_replay_is_bit_exact(prec):
    a = _run(prec, 12, graph=True)
    b = _run(prec, 12, graph=False)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_trajectory_shards_reproduce_one_run(prec):
    # trajectories [40, 70) run alone with traj_offset 40 equal rows 40..69 of the full run
    full = _run(prec, 6, graph=True, M=70)
    part = _run(prec, 6, graph=True, M=30, offset=40)
    for u, v in zip(full, part):
        assert np.array_equal(u[40:], v)


def test_profile_counts_launches():
    from paper_2608_10075_b300 import twa
    with twa.TWA(300, 1.0, 20.0, 1.0, 1e-3, precision="bf16x3") as g:
        g.run(130, 1)
        g.profile(True)
        g.run(130, 4)
        p = g.profile_read()
        g.profile(False)
    for k in ("noise", "predict", "correct", "close"):
        assert p[k][1] == 4 and p[k][0] > 0.0
    # the L.eta tiles of step t + 1 ride in the predictor and corrector launches of
    # step t; the first step of the run computed its own noise part already
    assert p["noise_factor"][1] == 0
    assert p["gemm64"][1] == 0
    # algorithmic FLOPs: all of W twice and the lower triangle of L once per step,
    # three BF16 products per W entry and two per L entry
    N, M = 300, 130
    w = 2.0 * N * N * 2 * M * 3
    l_tri = 2.0 * (N * (N + 1) / 2) * 2 * M * 2
    total = p["predict"][2] + p["correct"][2]
    assert abs(total - 4 * (2 * w + l_tri)) <= 1e-9 * total
    assert p["predict"][2] >= 4 * w and p["correct"][2] >= 4 * w


def test_profile_standalone_noise_factor_after_set_state():
    # a new state drops the precomputed noise part: one standalone L.eta launch
    from paper_2608_10075_b300 import twa
    with twa.TWA(300, 1.0, 20.0, 1.0, 1e-3, precision="bf16x3") as g:
        g.run(130, 2)
        s = g.get_state()
        g.set_state(*s)
        g.profile(True)
        g.run(130, 3)
        p = g.profile_read()
        g.profile(False)
    assert p["noise_factor"][1] == 1 and p["noise"][1] == 4 and p["predict"][1] == 3
    N, M = 300, 130
    assert abs(p["noise_factor"][2] - 2.0 * (N * (N + 1) / 2) * 2 * M * 2) <= 1e-9 * p["noise_factor"][2]


@pytest.mark.parametrize("prec,route,noise", [("fp64", "dense", "cholesky"), ("bf16x3", "dense", "cholesky"),
                                              ("bf16", "dense", "cholesky"), ("bf16x3", "fft", "circulant")])
def test_sample_stride_selects_every_kth_window_step(prec, route, noise):
    # window start n_w = 2, stride 3, 11 steps: samples after steps 5, 8, 11. The
    # library's window means must be the means of the collective moments of the
    # states read back after exactly those steps.
    from paper_2608_10075_b300 import twa
    N, M, steps, nw, k, dt = 50, 8, 11, 2, 3, 1e-3
    acc, n = np.zeros((M, 5)), 0
    with twa.TWA(N, 1.0, 8.0, 1.0, dt, seed=6, precision=prec, window_start=nw * dt, ws_route=route,
                 noise_route=noise, sample_stride=k) as g:
        for t in range(1, steps + 1):
            g.run(M, 1)
            if t > nw and (t - nw) % k == 0:
                x, y, z = g.get_state()
                Sx, Sy, Sz = x.sum(1), y.sum(1), z.sum(1)
                A = 0.25 * (Sx * Sx + Sy * Sy)
                acc += np.stack([Sz, A, A * A, A * Sz, Sz * Sz], axis=1)
                n += 1
        mom = g.moments()
        assert g.observables()["samples"] == n == 3
    # FP64 path: the same sums; mixed paths: FP32 state summed in a different order
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.allclose(mom, acc / n, rtol=tol, atol=tol * np.abs(acc / n).max())
