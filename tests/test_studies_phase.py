"""Host logic of the phase-diagram study (CPU): the pump prefactor from a target
w~ = w_max / (Gamma N), and the per-(N, alpha) summaries, checked with a fake
batch runner whose w_max is linear in w as the library's is."""
import argparse
import math

import numpy as np

from paper_2608_10075_b300 import studies


def _fake_runner(calls):
    def run(points, M, seed=0, precision="bf16x3", ws_route="dense"):
        calls.append((points, M))
        res = []
        for p in points:
            wmax = p["w"] * (1.0 + p["alpha"]) * math.sqrt(p["N"])        # any law linear in w
            wt = wmax / (p["Gamma"] * p["N"])
            g2 = 1.0 + (math.log10(wt) - 0.3 * p["alpha"]) ** 2          # minimum at w~ = 10^(0.3 alpha)
            res.append(dict(w_max=wmax, w_tilde=wt, g2=g2, g2_se=0.01, SpSm=p["N"] * 2.0 * wt,
                            sigma_z=-0.5, stability=0.1))
        return res, (256, 1)
    return run


def test_phase_study_sets_w_from_the_target_and_finds_the_minimum(capsys):
    args = argparse.Namespace(Ns=[100, 300], alphas=[0.5, 1.0], n_wt=21, wt_min=0.1, wt_max=10.0, M=64, T=1.0,
                              window=0.5, dt_scale=0.02, precision="bf16x3", spacing="log")
    calls = []
    studies.phase_study(args, runner=_fake_runner(calls))
    cal, grid = calls[0][0], calls[1][0]
    assert all(p["w"] == 1.0 and p["steps"] == 1 for p in cal) and len(cal) == 4
    assert len(grid) == 4 * 21 and calls[1][1] == 64
    assert all(p["steps"] == int(round(1.0 / (0.02 / p["N"]))) for p in grid)
    lines = [__import__("json").loads(x) for x in capsys.readouterr().out.strip().splitlines()]
    assert len(lines) == 4
    wts = np.logspace(-1, 1, 21)
    for d in lines:
        # the library's w~ of every point equals its target
        assert np.allclose(d["wt_lib"], wts, rtol=1e-12) and np.allclose(d["wt"], wts, rtol=1e-12)
        j = int(np.argmin([(math.log10(w) - 0.3 * d["alpha"]) ** 2 for w in wts]))
        assert d["wt_at_min"] == d["wt"][j] and d["g2_min"] == min(d["g2"])
        assert d["superradiant_wt"] == [w for w in d["wt"] if 2.0 * w > 1.0]


def test_phase_study_default_protocol_is_ten_equally_spaced_values(capsys):
    # ten equally spaced w~ in [1/10, 1]
    args = argparse.Namespace(Ns=[100], alphas=[0.7], n_wt=10, wt_min=0.1, wt_max=1.0, M=8, T=15.0, window=5.0,
                              dt_scale=0.02, precision="bf16x3", spacing="linear")
    calls = []
    studies.phase_study(args, runner=_fake_runner(calls))
    d = __import__("json").loads(capsys.readouterr().out.strip())
    assert np.allclose(d["wt"], np.arange(1, 11) / 10.0, rtol=1e-12)
    assert all(abs(p["window_start"] - 10.0) < 1e-9 for p in calls[1][0])
