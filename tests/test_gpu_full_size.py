"""The benchmark's qualifier at full size: mixed precision against the FP64 GPU
path, observables within 3 standard errors, at N = 10^4.

Workload of the benchmark (N = 10^4, alpha = 1, w = N Gamma / 2, Gamma = 1,
dt = 2e-5) on a subset of its ensemble: trajectories 0..127 (the same Philox
counters, so the same trajectories the benchmark integrates) over 400 steps,
window over the last 200. BF16X3 and FP64 run on the same seeds, so besides
the unpaired comparison (each side's standard error) the per-trajectory paired
differences show the precision error directly: it must be a small fraction of
the statistical error the observables are quoted with.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, ALPHA, W, GAMMA, DT = 10000, 1.0, 5000.0, 1.0, 2e-5


def _samples(means):
    """Per-trajectory samples of <S^z>, <S+S-> and <S+S+S-S-> (Sec. S1, items 5-6)."""
    Sz, A, A2, ASz, Sz2 = means.T
    return {"Sz": Sz, "SpSm": A + 0.5 * Sz, "G2num": A2 + 2 * ASz - Sz / 3 + 0.5 * Sz2 - 4.0 / 3.0 * A}


_RUNS = {}


def _run(prec, M=128, steps=400):
    from paper_2608_10075_b300 import twa
    if prec not in _RUNS:
        with twa.TWA(N, ALPHA, W, GAMMA, DT, seed=0, precision=prec, window_start=(steps // 2) * DT) as g:
            g.run(M, steps)
            _RUNS[prec] = (g.observables(), _samples(g.moments()))
    return _RUNS[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x2", "bf16b"])
def test_mixed_matches_fp64_gpu_at_n1e4(prec):
    M = 128
    obs, smp = {}, {}
    for p in (prec, "fp64"):
        obs[p], smp[p] = _run(p)
        assert obs[p]["samples"] == 200 and obs[p]["nonfinite"] == 0
    a, b = obs[prec], obs["fp64"]
    for k in ("Sz", "SpSm", "G2num", "g2"):
        se = math.hypot(a[k + "_se"], b[k + "_se"])
        assert abs(a[k] - b[k]) <= 3.0 * se, (k, a[k], b[k], se)
    for k in ("Sz", "SpSm", "G2num"):
        d = smp[prec][k] - smp["fp64"][k]
        paired, paired_se = float(np.mean(d)), float(np.std(d, ddof=1) / math.sqrt(M))
        unpaired_se = math.hypot(a[k + "_se"], b[k + "_se"])
        # the precision error is a small fraction of the statistical error
        assert abs(paired) + 3.0 * paired_se <= 0.1 * unpaired_se, (k, paired, paired_se, unpaired_se)
