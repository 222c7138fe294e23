"""Parity of the semi-implicit midpoint integrator (TWA_INT_MIDPOINT) with the
FP64 CPU oracle, through the C ABI.

The FP64 GPU path integrates the same discretised SDE as the oracle from the
same Philox stream, so every trajectory agrees to rounding (1e-9 relative over
200 steps). The tensor-core path keeps the Heun path's bounds: BF16X3 within
1e-2 and FP32 (TF32 hi/lo split) within 1e-4 of the oracle over three steps,
observables within 3 standard errors. Each stage is an exact rotation, so
spin lengths hold without renormalisation up to rounding.
"""
import math
import os

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle, pump_matrix

pytestmark = pytest.mark.gpu


def _twa():
    from paper_2608_10075_b300 import twa
    return twa


def _err(g, o):
    gx, gy, gz = g.get_state()
    return max(np.max(np.abs(gx - o.sx)), np.max(np.abs(gy - o.sy)), np.max(np.abs(gz - o.sz)))


@pytest.mark.parametrize("N,M,alpha,w,renorm", [(16, 64, 1.0, 8.0, True), (130, 40, 0.5, 30.0, True),
                                                 (37, 9, 2.0, 5.0, False), (1, 16, 1.0, 8.0, True),
                                                 (12, 8, 0.0, 3.0, True), (12, 8, math.inf, 3.0, False)])
def test_fp64_path_per_trajectory(N, M, alpha, w, renorm):
    twa = _twa()
    G, dt = 1.0, 2e-3
    o = TWAOracle(N, alpha, w, G, dt, 3, M, integrator="midpoint", renormalize=renorm)
    with twa.TWA(N, alpha, w, G, dt, seed=3, integrator="midpoint", renormalize=renorm) as g:
        for _ in range(4):
            o.run(50)
            g.run(M, 50)
            assert _err(g, o) <= 1e-9
        if not renorm:
            gx, gy, gz = g.get_state()
            assert np.max(np.abs(gx ** 2 + gy ** 2 + gz ** 2 - 3.0)) < 1e-11


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-2), ("bf16", 3e-2), ("fp32", 1e-4), ("tf32", 1e-2)])
@pytest.mark.parametrize("N,M", [(300, 200), (45, 3)])
def test_tensor_core_path_tracks_oracle(prec, tol, N, M):
    twa = _twa()
    alpha, w, G, dt = 1.0, 8.0, 1.0, 2e-3
    o = TWAOracle(N, alpha, w, G, dt, 11, M, integrator="midpoint")
    with twa.TWA(N, alpha, w, G, dt, seed=11, precision=prec, integrator="midpoint") as g:
        for _ in range(3):
            o.run(1)
            g.run(M, 1)
            assert _err(g, o) < tol


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_tensor_core_path_keeps_lengths_without_renormalisation(prec):
    # FP32 state: each rotation is exact up to a few roundings of 2^-24
    twa = _twa()
    with twa.TWA(200, 1.0, 20.0, 1.0, 1e-3, seed=2, precision=prec, integrator="midpoint",
                 renormalize=False) as g:
        g.run(64, 100)
        gx, gy, gz = g.get_state()
    assert np.max(np.abs(gx ** 2 + gy ** 2 + gz ** 2 - 3.0)) < 1e-4


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
@pytest.mark.parametrize("N,M,steps", [(200, 70, 7), (37, 5, 5)])
def test_mixed_launches_equal_separate_launches(prec, N, M, steps):
    twa = _twa()
    out = []
    old = os.environ.pop("TWA_SEPARATE_LETA", None)
    try:
        for sep in (False, True):
            if sep:
                os.environ["TWA_SEPARATE_LETA"] = "1"
            with twa.TWA(N, 1.0, 10.0, 1.0, 1e-3, seed=4, precision=prec, integrator="midpoint") as g:
                g.run(M, steps)
                out.append(g.get_state())
    finally:
        os.environ.pop("TWA_SEPARATE_LETA", None)
        if old is not None:
            os.environ["TWA_SEPARATE_LETA"] = old
    for u, v in zip(*out):
        assert np.array_equal(u, v)


def test_ensemble_observables_within_3se():
    N, alpha, w, G, dt, M, steps, t0 = 128, 1.0, 16.0, 1.0, 1e-3, 512, 1000, 0.5
    twa = _twa()
    o = TWAOracle(N, alpha, w, G, dt, 5, M, window_start=t0, integrator="midpoint")
    o.run(steps)
    ob = o.observables()
    for prec in ("bf16x3", "fp64"):
        with twa.TWA(N, alpha, w, G, dt, seed=5, precision=prec, window_start=t0, integrator="midpoint") as g:
            g.run(M, steps)
            gb = g.observables()
        for k in ("Sz", "SpSm", "G2num", "g2"):
            assert abs(gb[k] - ob[k]) <= 3.0 * math.hypot(gb[k + "_se"], ob[k + "_se"]), (prec, k, gb[k], ob[k])
        assert gb["nonfinite"] == 0


def test_full_size_sampled_trajectories():
    # N = 10^4, alpha = 1, w = N/2, dt = 2e-5, M = 1024 in the launch shape of the
    # benchmark; three trajectories recomputed one by one by the oracle
    twa = _twa()
    N, alpha, w, G, dt, M = 10000, 1.0, 5000.0, 1.0, 2e-5, 1024
    with twa.TWA(N, alpha, w, G, dt, seed=0, precision="bf16x3", integrator="midpoint") as g:
        g.run(M, 2)
        gx, gy, gz = g.get_state()
    W = pump_matrix(N, alpha, w)
    L = np.linalg.cholesky(W)
    for m in (0, 517, 1023):
        o = TWAOracle(N, alpha, w, G, dt, 0, 1, m0=m, W=W, L=L, integrator="midpoint")
        o.run(2)
        err = max(np.max(np.abs(gx[m] - o.sx[0])), np.max(np.abs(gy[m] - o.sy[0])), np.max(np.abs(gz[m] - o.sz[0])))
        assert err < 1e-2, (m, err)


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-2), ("fp32", 1e-3)])
@pytest.mark.parametrize("noise", ["cholesky", "circulant"])
def test_fft_route(prec, tol, noise):
    # W.s by the circulant FFT, the midpoint state as the second transform's input
    twa = _twa()
    N, M, alpha, w, G, dt = 300, 40, 1.0, 8.0, 1.0, 2e-3
    if noise == "cholesky":
        o = TWAOracle(N, alpha, w, G, dt, 11, M, integrator="midpoint")
    else:
        from oracle.circulant import TWAOracleCirculant
        o = TWAOracleCirculant(N, alpha, w, G, dt, 11, M, integrator="midpoint")
    with twa.TWA(N, alpha, w, G, dt, seed=11, precision=prec, ws_route="fft", noise_route=noise,
                 integrator="midpoint") as g:
        for _ in range(3):
            o.run(1)
            g.run(M, 1)
            assert _err(g, o) < tol
    with twa.TWA(N, alpha, w, G, dt, seed=11, precision=prec, ws_route="fft", noise_route=noise,
                 integrator="midpoint", renormalize=False) as g:
        g.run(M, 100)
        gx, gy, gz = g.get_state()
    assert np.max(np.abs(gx ** 2 + gy ** 2 + gz ** 2 - 3.0)) < 1e-4


def test_rejections():
    twa = _twa()
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, integrator=2)
    assert e.value.name == "TWA_EINVAL"
    with twa.TWA(32, 1.0, 8.0, 1.0, 1e-3, integrator="midpoint") as g:
        with pytest.raises(twa.TWAError) as e:
            g.grad("SpSm", 8, 4)
        assert e.value.name == "TWA_EUNSUPPORTED"
