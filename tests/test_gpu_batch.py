"""Batched scans (twa_batch_run) through the C ABI.

Against the oracle: every point's per-trajectory window means over its first
steps follow the oracle run on the same BF16-rounded normals within the bound
derived in tests/mixed_bounds.py, and after a windowed run each point's
observables lie within 3 standard errors of the plain FP64 oracle's.

Every point of a batch runs the same kernels, with the same tile arithmetic,
as when it runs alone: a tile's accumulation order along K does not depend on
the K-stage width, the per-site results do not depend on the trajectory-tile
width, and the collective sums are formed per 128-site row tile in a fixed
order. So each point's observables must equal its standalone twa_run result,
whatever tile configuration the autotuner picks.
"""
import math
import os

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle
from tests.mixed_bounds import BF16NoiseOracle, step_bound

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
        assert cfg in ((256, 1), (192, 1), (256, 0), (128, 1))   # BF16X3: no six-stage candidate
    for p, r in zip(POINTS, res):
        ref = _alone(p, M, seed)
        assert r["steps"] == p["steps"] and r["samples"] == ref["samples"]
        for k in ("Sz", "SpSm", "G2num", "g2", "Sz_se", "g2_se"):
            assert abs(r[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (p, k, r[k], ref[k])
        assert math.isfinite(r["w_max"]) and r["nonfinite"] == 0


@pytest.mark.parametrize("prec", ["bf16x2", "bf16l2", "bf16b"])
def test_batch_in_the_two_product_precisions_equals_points_run_alone(prec):
    from paper_2608_10075_b300 import twa
    M, seed = 64, 5
    # N = 700: rows whose W (and, in BF16B, L) lie mostly off the two-product band
    pts = POINTS + ([dict(N=700, alpha=1.0, w=350.0, Gamma=1.0, dt=1e-4, steps=20, window_start=0.001)]
                    if prec != "bf16x2" else [])
    res, _ = twa.batch_run(pts, M, seed=seed, precision=prec)
    for p, r in zip(pts, res):
        with twa.TWA(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed=seed, precision=prec,
                     window_start=p["window_start"]) as g:
            g.run(M, p["steps"])
            ref = g.observables()
        for k in ("Sz", "SpSm", "G2num", "g2", "Sz_se", "g2_se"):
            assert abs(r[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (p, k, r[k], ref[k])


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


# uneven points: ragged N (37, 130, 300), the extreme exponents of the scans
ORACLE_POINTS = [
    dict(N=300, alpha=0.25, w=60.0, Gamma=1.0, dt=2e-4),
    dict(N=37, alpha=1.0, w=3.0, Gamma=1.0, dt=1e-3),
    dict(N=130, alpha=2.0, w=10.0, Gamma=1.0, dt=3e-4),
    dict(N=200, alpha=0.5, w=100.0, Gamma=1.0, dt=1e-4),
]


def _moment_bound(o, D):
    """Bound of the window-moment samples (S^z, A, A^2, A S^z, (S^z)^2) of the
    oracle's current state when every collective sum S^a may be off by D[m]."""
    Sx, Sy, Sz = o.sx.sum(1), o.sy.sum(1), o.sz.sum(1)
    A = 0.25 * (Sx * Sx + Sy * Sy)
    dA = 0.5 * (np.abs(Sx) + np.abs(Sy)) * D + 0.5 * D * D
    return np.stack([D, dA, 2 * np.abs(A) * dA + dA * dA, np.abs(A) * D + np.abs(Sz) * dA + dA * D,
                     2 * np.abs(Sz) * D + D * D], axis=1)


def test_batch_points_track_the_oracle_per_trajectory():
    from paper_2608_10075_b300 import twa
    M, seed, steps = 160, 3, 3
    pts = [dict(p, steps=steps, window_start=0.0) for p in ORACLE_POINTS]
    res, _ = twa.batch_run(pts, M, seed=seed, means=True)
    for p, r in zip(pts, res):
        o = BF16NoiseOracle(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed, M)
        tol = 0.0
        mbound = np.zeros((M, 5))
        for _ in range(steps):
            tol = tol + step_bound(o, o.sx, o.sy, o.sz)
            o.run(1)
            # state differences <= 2 x the summed step bounds (tests/mixed_bounds.py),
            # summed over sites; the kernel forms S^a in FP32 (N 2^-23 sqrt 3 more)
            D = (2.0 * tol).sum(axis=1) + p["N"] * 2.0 ** -23 * math.sqrt(3.0)
            mbound += _moment_bound(o, D)
        mbound /= steps
        ref = o.window_means()
        err = np.abs(r["means"] - ref)
        assert np.all(err <= mbound), (p, float(np.max(err / mbound)))
        assert r["samples"] == steps and r["nonfinite"] == 0


def test_batch_observables_within_3se_of_the_oracle():
    from paper_2608_10075_b300 import twa
    M, seed, steps = 256, 21, 400
    pts = [dict(p, steps=steps, window_start=0.5 * steps * p["dt"]) for p in ORACLE_POINTS]
    res, _ = twa.batch_run(pts, M, seed=seed)
    for p, r in zip(pts, res):
        o = TWAOracle(p["N"], p["alpha"], p["w"], p["Gamma"], p["dt"], seed, M, window_start=p["window_start"])
        o.run(steps)
        ob = o.observables()
        for k in ("Sz", "SpSm", "G2num", "g2"):
            assert abs(r[k] - ob[k]) <= 3.0 * math.hypot(r[k + "_se"], ob[k + "_se"]), (p, k, r[k], ob[k])
