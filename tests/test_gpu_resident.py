"""The resident route (ws_route = TWA_ROUTE_RESIDENT, FP32 SIMT, whole run in
one launch) against the FP64 oracle, through the C ABI.

Its arithmetic is FP32 throughout with the FP32 Box-Muller normals of the mixed
paths (which differ from the oracle's FP64 normals by ~1e-6 relative), so a
trajectory follows the oracle's to ~1e-5 over a few steps (as the FP32 mode of
the tensor-core path); beyond that the comparison is statistical. Sizes cover
every CTA shape (8 to 64 trajectories per CTA), W and L held in shared memory
(small N) and streamed through it (large N), and ragged trajectory counts.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle

pytestmark = pytest.mark.gpu


def _twa():
    from paper_2608_10075_b300 import twa
    return twa


@pytest.mark.parametrize("integrator", ["heun", "midpoint"])
@pytest.mark.parametrize("N,M", [(16, 70), (37, 37), (100, 65), (130, 33), (300, 17), (512, 9)])
def test_trajectories_track_the_oracle(N, M, integrator):
    twa = _twa()
    alpha, w, G, dt = 1.0, 8.0, 1.0, 2e-3
    o = TWAOracle(N, alpha, w, G, dt, 13, M, integrator=integrator)
    with twa.TWA(N, alpha, w, G, dt, seed=13, precision="fp32", ws_route="resident", integrator=integrator) as g:
        for k in (1, 2, 5):
            o.run(k)
            g.run(M, k)   # one launch per call
            gx, gy, gz = g.get_state()
            err = max(np.max(np.abs(gx - o.sx)), np.max(np.abs(gy - o.sy)), np.max(np.abs(gz - o.sz)))
            assert err < 1e-4, (k, err)
            assert np.max(np.abs(gx ** 2 + gy ** 2 + gz ** 2 - 3.0)) < 5e-6


def test_continuation_is_exact():
    # 5 + 7 steps in two launches equal 12 steps in one, bit for bit
    twa = _twa()
    N, M = 90, 40
    out = []
    for parts in ((12,), (5, 7)):
        with twa.TWA(N, 1.0, 6.0, 1.0, 1e-3, seed=2, precision="fp32", ws_route="resident",
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
    with twa.TWA(N, alpha, w, G, dt, seed=5, precision="fp32", ws_route="resident", window_start=t0) as g:
        g.run(M, steps)
        gb = g.observables()
    assert gb["samples"] == steps // 2
    for k in ("Sz", "SpSm", "G2num", "g2"):
        assert abs(gb[k] - ob[k]) <= 3.0 * math.hypot(gb[k + "_se"], ob[k + "_se"]), (k, gb[k], ob[k])
    assert gb["nonfinite"] == 0


POINTS = [
    dict(N=300, alpha=0.25, w=60.0, Gamma=1.0, dt=2e-4, steps=150, window_start=0.015),
    dict(N=37, alpha=1.0, w=3.0, Gamma=1.0, dt=1e-3, steps=400, window_start=0.2),
    dict(N=100, alpha=2.0, w=10.0, Gamma=1.0, dt=3e-4, steps=250, window_start=0.0375),
    dict(N=512, alpha=0.5, w=100.0, Gamma=1.0, dt=1e-4, steps=60, window_start=0.003),
]


def test_batch_equals_points_run_alone_and_the_oracle():
    twa = _twa()
    M, seed = 96, 17
    res, tiles = twa.batch_run(POINTS, M, seed=seed, precision="fp32", ws_route="resident", means=True)
    assert tiles == (0, 0)
    for p, r in zip(POINTS, res):
        with twa.TWA(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed=seed, precision="fp32",
                     ws_route="resident", window_start=p["window_start"]) as g:
            g.run(M, p["steps"])
            ref = g.observables()
            mom = g.moments()
        assert np.array_equal(r["means"], mom), p
        for k in ("Sz", "SpSm", "G2num", "g2", "Sz_se", "g2_se"):
            assert abs(r[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (p, k, r[k], ref[k])
        o = TWAOracle(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed, M, window_start=p["window_start"])
        o.run(p["steps"])
        ob = o.observables()
        for k in ("Sz", "SpSm", "G2num", "g2"):
            assert abs(r[k] - ob[k]) <= 3.0 * math.hypot(r[k + "_se"], ob[k + "_se"]), (p, k, r[k], ob[k])


def test_resident_route_rejections():
    twa = _twa()
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(513, 1.0, 8.0, 1.0, 1e-3, precision="fp32", ws_route="resident")
    assert e.value.name == "TWA_EUNSUPPORTED"
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="bf16x3", ws_route="resident")
    assert e.value.name == "TWA_EUNSUPPORTED"
    with pytest.raises(twa.TWAError) as e:
        twa.batch_run([dict(N=600, alpha=1.0, w=4.0, Gamma=1.0, dt=1e-3, steps=4)], 8, precision="fp32",
                      ws_route="resident")
    assert e.value.name == "TWA_EUNSUPPORTED"
