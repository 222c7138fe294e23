"""The phase-diagram workflow (studies.py phase) on the GPU against the oracle,
on a tiny grid: the pump prefactor it derives from each target w~ (one
calibration batch, w_max linear in w) must equal the oracle's spectrum, and
every point's g2, <S+S-> and sigma_z must lie within 3 standard errors of the
FP64 oracle run at that prefactor (same seed, same trajectories)."""
import argparse
import json
import math

import pytest

from oracle.twa_oracle import TWAOracle, spectrum

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,route", [("bf16x2", "dense"), ("fp32", "resident")])
def test_phase_study_matches_the_oracle(precision, route, capsys):
    from paper_2608_10075_b300 import studies
    N, alphas, wts, M, T, window, dt_scale = 24, [0.7, 2.0], [0.3, 1.0], 128, 1.0, 0.5, 0.02
    args = argparse.Namespace(Ns=[N], alphas=alphas, n_wt=len(wts), wt_min=wts[0], wt_max=wts[-1], M=M, T=T,
                              window=window, dt_scale=dt_scale, precision=precision, spacing="linear",
                              route=route)
    studies.phase_study(args)
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines() if x.startswith("{")]
    assert len(lines) == len(alphas)
    dt = dt_scale / N
    steps = int(round(T / dt))
    for d in lines:
        a = d["alpha"]
        wmax1 = spectrum(N, a, 1.0)[0]
        for k, wt in enumerate(d["wt"]):
            w = wt * N / wmax1
            assert abs(d["wt_lib"][k] - wt) <= 1e-6 * wt, (a, wt, d["wt_lib"][k])
            o = TWAOracle(N, a, w, 1.0, dt, 0, M, window_start=max(0.0, steps * dt - window))
            o.run(steps)
            ob = o.observables()
            g2, se = d["g2"][k], d["g2_se"][k]
            assert abs(g2 - ob["g2"]) <= 3.0 * math.hypot(se, ob["g2_se"]), (a, wt, g2, ob["g2"])
            assert abs(d["sigma_z"][k] - ob["sigma_z"]) <= 3.0 * (ob["sigma_z_se"] * math.sqrt(2.0)) + 1e-12
        assert d["g2_min"] == min(d["g2"])
