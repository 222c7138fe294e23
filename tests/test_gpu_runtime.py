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


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32", "fp32"])
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


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3", "bf16b", "fp32"])
def test_noise_draw_beside_the_launches_gives_the_same_bits(monkeypatch, prec, graph):
    # the noise of step t + 2 drawn by the epilogue threads of step t's two
    # launches (default for the BF16 precisions), on a second stream while they
    # run ("1": the FP32 precision's default), or on the context's stream before
    # them ("0"); with a continuation and a set_state in between (the noise is
    # primed again)
    from paper_2608_10075_b300 import twa
    out = {}
    for overlap in ("epi", "1", "0"):
        monkeypatch.setenv("TWA_NOISE_EPILOGUE", "1" if overlap == "epi" else "0")
        monkeypatch.setenv("TWA_NOISE_OVERLAP", "1" if overlap == "epi" else overlap)
        if not graph:
            monkeypatch.setenv("TWA_NO_GRAPH", "1")
        with twa.TWA(260, 1.0, 20.0, 1.0, 1e-3, seed=9, precision=prec, window_start=0.004) as g:
            g.run(70, 7)
            g.run(70, 6)
            x, y, z = g.get_state()
            g.set_state(x, y, z)
            g.run(70, 5)
            out[overlap] = (g.get_state(), g.observables())
    for mode in ("1", "0"):
        for u, v in zip(out["epi"][0], out[mode][0]):
            assert np.array_equal(u, v), mode
        for k in ("Sz", "SpSm", "G2num", "g2"):
            assert out["epi"][1][k] == out[mode][1][k], (mode, k)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_trajectory_shards_reproduce_one_run(prec):
    # trajectories [40, 70) run alone with traj_offset 40 equal rows 40..69 of the full run
    full = _run(prec, 6, graph=True, M=70)
    part = _run(prec, 6, graph=True, M=30, offset=40)
    for u, v in zip(full, part):
        assert np.array_equal(u[40:], v)


def test_profile_counts_launches(monkeypatch):
    # the noise draw as its own kernel (TWA_NOISE_EPILOGUE=0), serial when profiling
    monkeypatch.setenv("TWA_NOISE_EPILOGUE", "0")
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
    # and the algorithmic count: the same products counted once
    alg = p["predict"][3] + p["correct"][3]
    assert abs(alg - 4 * (2 * w / 3 + l_tri / 2)) <= 1e-9 * alg


def test_noise_drawn_inside_the_launches():
    # by default the BF16 precisions' dense step has no noise kernel: the two
    # launches of step t draw the noise of step t + 2 (the prime of a run draws
    # steps t and t + 1 as before)
    from paper_2608_10075_b300 import twa
    with twa.TWA(300, 1.0, 20.0, 1.0, 1e-3, precision="bf16b") as g:
        g.run(130, 1)
        g.profile(True)
        g.run(130, 4)
        p = g.profile_read()
        g.profile(False)
    assert p["noise"][1] == 0
    assert p["predict"][1] == 4 and p["correct"][1] == 4 and p["close"][1] == 4


def test_profile_counts_the_two_product_band():
    # BF16B at N = 1000 (four 256-row units): every W entry one product, plus a
    # second over the K columns [u - 64, u + 320) of each unit's rows; L the
    # same over its lower triangle, the band's stages counted in full
    from paper_2608_10075_b300 import twa
    N, M = 1000, 64
    with twa.TWA(N, 1.0, 20.0, 1.0, 1e-3, precision="bf16b") as g:
        g.run(M, 1)
        g.profile(True)
        g.run(M, 2)
        p = g.profile_read()
        g.profile(False)
    cols = 2 * M
    w_alg = 2.0 * N * N * cols
    l_alg = 2.0 * (N * (N + 1) / 2) * cols
    band_w = sum(min(256, N - u) * (min(u + 320, N) - max(u - 64, 0)) for u in range(0, N, 256))
    band_l = sum(min(256, N - u) * (min(u + 256, N) - max(u - 64, 0)) for u in range(0, N, 256))
    alg = p["predict"][3] + p["correct"][3]
    issued = p["predict"][2] + p["correct"][2]
    assert abs(alg - 2 * (2 * w_alg + l_alg)) <= 1e-9 * alg
    want = 2 * (2 * (w_alg + 2.0 * band_w * cols) + l_alg + 2.0 * band_l * cols)
    assert abs(issued - want) <= 1e-9 * issued, (issued, want)


def test_profile_standalone_noise_factor_after_set_state(monkeypatch):
    # a new state drops the precomputed noise part: one standalone L.eta launch
    monkeypatch.setenv("TWA_NOISE_EPILOGUE", "0")
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


def _count_allocator():
    """(alloc, free) over torch's caching allocator that record every pointer."""
    import torch
    live, log = {}, {"alloc": 0, "free": 0, "bad_free": 0}

    def alloc(nbytes, stream):
        p = torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
        live[p] = nbytes
        log["alloc"] += 1
        return p

    def free(ptr, stream):
        if live.pop(ptr, None) is None:
            log["bad_free"] += 1
        log["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    return (alloc, free), live, log


@pytest.mark.parametrize("prec,route,noise", [("fp64", "dense", "cholesky"), ("bf16x3", "dense", "cholesky"),
                                              ("bf16x3", "fft", "circulant")])
def test_caller_allocator_gives_the_same_results_and_frees_everything(prec, route, noise):
    # all device memory of the context and of its calls from the caller's
    # allocator (here torch's caching allocator): same bits as the library's own
    # allocator, every block handed back exactly once by twa_destroy
    import torch
    from paper_2608_10075_b300 import twa
    N, M, steps = 130, 40, 7
    kw = dict(seed=5, precision=prec, window_start=0.002, ws_route=route, noise_route=noise)
    with twa.TWA(N, 1.0, 12.0, 1.0, 1e-3, **kw) as g:
        g.run(M, steps)
        ref = g.get_state()
        ref_obs = g.observables()
    base = torch.cuda.memory_allocated()
    pair, live, log = _count_allocator()
    with twa.TWA(N, 1.0, 12.0, 1.0, 1e-3, allocator=pair, **kw) as g:
        g.run(M, steps)
        st = g.get_state()
        obs = g.observables()
        assert torch.cuda.memory_allocated() - base >= sum(live.values()) >= 2 * 8 * N * N   # W, L in FP64
    for a, b in zip(ref, st):
        assert np.array_equal(a, b)
    for k in ("Sz", "SpSm", "G2num", "g2"):
        assert obs[k] == ref_obs[k]
    assert log["alloc"] > 0 and log["alloc"] == log["free"] and log["bad_free"] == 0 and not live
    assert torch.cuda.memory_allocated() == base


def test_caller_allocator_in_gradients_and_batches():
    import torch
    from paper_2608_10075_b300 import twa
    base = torch.cuda.memory_allocated()
    pair, live, log = _count_allocator()
    with twa.TWA(40, 0.8, 10.0, 1.0, 1e-3, seed=2, precision="fp64", window_start=0.01, allocator=pair) as g:
        r1 = g.grad("g2", 24, 30, checkpoint=7)
    with twa.TWA(40, 0.8, 10.0, 1.0, 1e-3, seed=2, precision="fp64", window_start=0.01) as g:
        r0 = g.grad("g2", 24, 30, checkpoint=7)
    assert r1["dJ_dw"] == r0["dJ_dw"] and r1["dJ_dalpha"] == r0["dJ_dalpha"]
    pts = [dict(N=100, alpha=1.5, w=25.0, Gamma=1.0, dt=5e-4, steps=9, window_start=0.001),
           dict(N=37, alpha=1.0, w=3.0, Gamma=1.0, dt=1e-3, steps=6, window_start=0.002)]
    a, _ = twa.batch_run(pts, 16, seed=3, allocator=pair)
    b, _ = twa.batch_run(pts, 16, seed=3)
    for x, y in zip(a, b):
        for k in ("Sz", "SpSm", "G2num", "g2"):
            assert x[k] == y[k]
    assert log["alloc"] == log["free"] and log["bad_free"] == 0 and not live
    assert torch.cuda.memory_allocated() == base


@pytest.mark.parametrize("prec", ["bf16x2", "fp32"])
def test_fp32_state_calls_match_the_fp64_ones(prec):
    # twa_get_state_f32 / twa_set_state_f32 move the FP32 state as it is: the
    # FP64 calls see the same values widened, and a run continued from either
    # gives the same bits (host and device buffers)
    import torch
    from paper_2608_10075_b300 import twa
    kw = dict(seed=6, precision=prec, window_start=0.002)
    with twa.TWA(150, 1.0, 20.0, 1.0, 1e-3, **kw) as g:
        g.run(40, 5)
        a = g.get_state_f32()
        b = g.get_state()
        for u, v in zip(a, b):
            assert u.dtype == np.float32 and np.array_equal(u.astype(np.float64), v)
        ad = g.get_state_f32(device="cuda")
        for u, v in zip(a, ad):
            assert np.array_equal(u, v.cpu().numpy())
    runs = []
    for state in (a, b, ad):
        with twa.TWA(150, 1.0, 20.0, 1.0, 1e-3, **kw) as g:
            g.set_state(*state)
            g.run(40, 6)
            runs.append((g.get_state(), g.observables()))
    for r in runs[1:]:
        for u, v in zip(runs[0][0], r[0]):
            assert np.array_equal(u, v)
        assert r[1]["SpSm"] == runs[0][1]["SpSm"]
    with twa.TWA(20, 1.0, 2.0, 1.0, 1e-3, precision="fp64") as g:
        g.run(4, 1)
        with pytest.raises(twa.TWAError) as e:
            g.get_state_f32()
        assert e.value.name == "TWA_EUNSUPPORTED"
        with pytest.raises(twa.TWAError) as e:
            g.set_state(*(np.zeros((4, 20), dtype=np.float32) for _ in range(3)))
        assert e.value.name == "TWA_EUNSUPPORTED"
