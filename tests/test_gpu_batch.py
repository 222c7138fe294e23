"""Batched scans (twa_batch_run) through the C ABI.

Every point of a batch runs the same kernels, with the same tile arithmetic,
as when it runs alone: a tile's accumulation order along K does not depend on
the K-stage width, the per-site results do not depend on the trajectory-tile
width, and the collective sums are formed per 128-site row tile in a fixed
order. So each point's observables must equal its standalone twa_run result,
whatever tile configuration the autotuner picks.
"""
import math
import os

import pytest

pytestmark = pytest.mark.gpu

POINTS = [
    dict(N=300, alpha=0.5, w=60.0, Gamma=1.0, dt=2e-4, steps=60, window_start=0.004),
    dict(N=100, alpha=1.5, w=25.0, Gamma=1.0, dt=5e-4, steps=25, window_start=0.005),
    dict(N=200, alpha=1.0, w=200.0, Gamma=1.0, dt=1e-4, steps=80, window_start=0.002),
    dict(N=130, alpha=2.0, w=10.0, Gamma=1.0, dt=3e-4, steps=60, window_start=0.009),
    dict(N=300, alpha=0.25, w=300.0, Gamma=1.0, dt=1e-4, steps=25, window_start=0.001),
    dict(N=37, alpha=1.0, w=3.0, Gamma=1.0, dt=1e-3, steps=80, window_start=0.02),
]


def _alone(p, M, seed, integrator="heun"):
    from paper_2608_10075_b300 import twa
    with twa.TWA(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed=seed, precision="bf16x3",
                 window_start=p["window_start"], integrator=integrator) as g:
        g.run(M, p["steps"])
        return g.observables()


@pytest.mark.parametrize("tiles", [None, ("192", "0")])
def test_batch_equals_points_run_alone(tiles):
    from paper_2608_10075_b300 import twa
    M, seed = 96, 11
    old = {k: os.environ.get(k) for k in ("TWA_TC_BN", "TWA_TC_KC")}
    if tiles:
        os.environ["TWA_TC_BN"], os.environ["TWA_TC_KC"] = tiles
    try:
        res, cfg = twa.batch_run(POINTS, M, seed=seed)
    finally:
        for k, v in old.items():
            os.environ.pop(k, None)
            if v is not None:
                os.environ[k] = v
    if tiles:
        assert cfg == (int(tiles[0]), int(tiles[1]))
    else:
        assert cfg in ((256, 1), (192, 1), (256, 0), (128, 1))
    for p, r in zip(POINTS, res):
        ref = _alone(p, M, seed)
        assert r["steps"] == p["steps"] and r["samples"] == ref["samples"]
        for k in ("Sz", "SpSm", "G2num", "g2", "Sz_se", "g2_se"):
            assert abs(r[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (p, k, r[k], ref[k])
        assert math.isfinite(r["w_max"]) and r["nonfinite"] == 0


def test_batch_with_the_midpoint_integrator_equals_points_run_alone():
    # the midpoint scheme's descriptors (corrector rotating s in place, predictor
    # writing the midpoint images) inside one batched plan
    from paper_2608_10075_b300 import twa
    M, seed = 64, 7
    res, _ = twa.batch_run(POINTS, M, seed=seed, integrator="midpoint")
    for p, r in zip(POINTS, res):
        ref = _alone(p, M, seed, integrator="midpoint")
        for k in ("Sz", "SpSm", "G2num", "g2", "Sz_se", "g2_se"):
            assert abs(r[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (p, k, r[k], ref[k])
        assert r["nonfinite"] == 0


def test_batch_rejects_fp64():
    from paper_2608_10075_b300 import twa
    with pytest.raises(twa.TWAError) as e:
        twa.batch_run(POINTS[:1], 8, precision="fp64")
    assert e.value.name == "TWA_EUNSUPPORTED"
