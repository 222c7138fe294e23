"""The resident route on the tensor cores (ws_route = TWA_ROUTE_RESIDENT with
precision BF16X2, N <= 128: W, L and the trajectory tile's operand images in
shared memory, accumulators in TMEM, the state in registers, a whole call in
one launch), through the C ABI.

Its arithmetic is that of the dense route's BF16X2 step: W and L as BF16 hi +
lo images (of W / w and L / sqrt(w)), the state and the noise rounded once to
BF16, FP32 accumulation and state. A trajectory is therefore checked against the
oracle run on the same BF16-rounded normals within the per-step bound derived
for BF16X2 (tests/mixed_bounds.py), and against the dense route itself, from
which it differs only in the order of the FP32 sums.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle

pytestmark = pytest.mark.gpu


def _twa():
    from paper_2608_10075_b300 import twa
    return twa


@pytest.mark.parametrize("N,M", [(16, 70), (37, 33), (64, 96), (100, 45), (128, 32)])
def test_trajectories_track_the_oracle_within_the_bf16x2_bound(N, M):
    from tests.mixed_bounds import BF16NoiseOracle, track
    twa = _twa()
    alpha, w, G, dt = 1.0, 8.0, 1.0, 2e-3
    o = BF16NoiseOracle(N, alpha, w, G, dt, 11, M)
    with twa.TWA(N, alpha, w, G, dt, seed=11, precision="bf16x2", ws_route="resident") as g:
        def step():
            g.run(M, 1)   # one launch per call
            return g.get_state()
        track(o, step, 3, "bf16x2")
        x, y, z = g.get_state()
    assert np.max(np.abs(x * x + y * y + z * z - 3.0)) < 5e-6


@pytest.mark.parametrize("integrator", ["heun", "midpoint"])
@pytest.mark.parametrize("N,M,alpha", [(20, 50, 1.0), (64, 64, 0.5), (101, 70, 2.0), (128, 40, 1.0)])
def test_matches_the_dense_route(N, M, alpha, integrator):
    # the same products (W, L hi + lo against BF16 operands) in another order
    # of the FP32 sums: the trajectories stay together to FP32 rounding
    twa = _twa()
    out = {}
    for route in ("dense", "resident"):
        with twa.TWA(N, alpha, 10.0, 1.0, 1e-3, seed=4, precision="bf16x2", ws_route=route,
                     integrator=integrator, window_start=0.01) as g:
            g.run(M, 20)
            out[route] = (g.get_state(), g.observables())
    err = max(np.max(np.abs(a - b)) for a, b in zip(out["dense"][0], out["resident"][0]))
    assert err < 1e-4, err
    for k in ("Sz", "SpSm", "g2"):
        a, b = out["dense"][1][k], out["resident"][1][k]
        assert abs(a - b) <= 1e-4 * abs(a), (k, a, b)


def test_continuation_is_exact():
    twa = _twa()
    N, M = 90, 70
    out = []
    for parts in ((12,), (5, 7)):
        with twa.TWA(N, 1.0, 6.0, 1.0, 1e-3, seed=2, precision="bf16x2", ws_route="resident",
                     window_start=0.004) as g:
            for p in parts:
                g.run(M, p)
            out.append((g.get_state(), g.moments()))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], out[1][1])


def test_observables_within_3se():
    twa = _twa()
    N, alpha, w, G, dt, M, steps, t0 = 64, 1.0, 16.0, 1.0, 1e-3, 512, 1000, 0.5
    o = TWAOracle(N, alpha, w, G, dt, 5, M, window_start=t0)
    o.run(steps)
    ob = o.observables()
    with twa.TWA(N, alpha, w, G, dt, seed=5, precision="bf16x2", ws_route="resident", window_start=t0) as g:
        g.run(M, steps)
        gb = g.observables()
    assert gb["samples"] == steps // 2
    for k in ("Sz", "SpSm", "G2num", "g2"):
        assert abs(gb[k] - ob[k]) <= 3.0 * math.hypot(gb[k + "_se"], ob[k + "_se"]), (k, gb[k], ob[k])
    assert gb["nonfinite"] == 0


POINTS = [
    dict(N=37, alpha=1.0, w=3.0, Gamma=1.0, dt=1e-3, steps=400, window_start=0.2),
    dict(N=100, alpha=2.0, w=10.0, Gamma=1.0, dt=3e-4, steps=250, window_start=0.0375),
    dict(N=128, alpha=0.5, w=40.0, Gamma=1.0, dt=2e-4, steps=120, window_start=0.012),
    dict(N=7, alpha=0.25, w=2.0, Gamma=1.0, dt=1e-3, steps=300, window_start=0.1),
]


def test_batch_equals_points_run_alone_and_the_oracle():
    twa = _twa()
    M, seed = 80, 17
    res, tiles = twa.batch_run(POINTS, M, seed=seed, precision="bf16x2", ws_route="resident", means=True)
    assert tiles == (0, 0)
    for p, r in zip(POINTS, res):
        with twa.TWA(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed=seed, precision="bf16x2",
                     ws_route="resident", window_start=p["window_start"]) as g:
            g.run(M, p["steps"])
            ref = g.observables()
            mom = g.moments()
        assert np.array_equal(r["means"], mom), p
        o = TWAOracle(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed, M, window_start=p["window_start"])
        o.run(p["steps"])
        ob = o.observables()
        for k in ("Sz", "SpSm", "G2num", "g2"):
            assert abs(r[k] - ob[k]) <= 3.0 * math.hypot(r[k + "_se"], ob[k + "_se"]), (p, k, r[k], ob[k])


def test_rejections():
    twa = _twa()
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(129, 1.0, 8.0, 1.0, 1e-3, precision="bf16x2", ws_route="resident")
    assert e.value.name == "TWA_EUNSUPPORTED"
    with pytest.raises(twa.TWAError) as e:
        twa.batch_run([dict(N=200, alpha=1.0, w=4.0, Gamma=1.0, dt=1e-3, steps=4)], 8, precision="bf16x2",
                      ws_route="resident")
    assert e.value.name == "TWA_EUNSUPPORTED"
