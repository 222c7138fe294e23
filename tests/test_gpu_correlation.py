"""Two-time correlations, spectrum and linewidth (twa_correlation) against the
FP64 oracle (oracle/two_time.py), through the C ABI.

FP64 path: the three copies reproduce the oracle's trajectories to rounding,
so every recorded lag's eight ensemble means, C(tau), S(omega) and the width
with its jackknife error agree to ~1e-9 relative. The responses are
differences of two nearby trajectories divided by eps, so their absolute error
is the trajectories' divided by eps; eps = 1e-3 keeps that far below 1e-9 of
their scale.

Mixed precision: C(tau) at every lag within 4 combined jackknife standard
errors of the oracle (many correlated lags: 4 rather than 3), the width within 3.
"""
import math

import numpy as np
import pytest

from oracle.two_time import two_time

pytestmark = pytest.mark.gpu


_REF = {}


def _reference(*args):
    # the mixed-precision cases share one oracle run
    if args not in _REF:
        _REF[args] = two_time(*args[:-2], _omegas(*args[-2:]))
    return _REF[args]


def _omegas(n, omax):
    return np.array([-omax + j * (2.0 * omax / (n - 1)) for j in range(n - 1)] + [omax])


def test_fp64_matches_the_oracle_lag_by_lag():
    from paper_2608_10075_b300 import twa
    N, alpha, w, G, dt, seed = 37, 1.0, 4.0, 1.0, 2e-3, 4
    M, prep, lags, stride, eps, n_om, omax = 64, 40, 600, 10, 1e-3, 321, 40.0
    ref = two_time(N, alpha, w, G, dt, seed, M, prep, lags, stride, eps, _omegas(n_om, omax))
    with twa.TWA(N, alpha, w, G, dt, seed=seed, precision="fp64") as g:
        got = g.correlation(M, prep, lags, stride, eps, n_om, omax)
    assert got["n_lags"] == ref["parts"].shape[0] == 61
    assert math.isfinite(ref["fwhm"]) and math.isfinite(ref["fwhm_se"])
    scale = np.max(np.abs(ref["parts"]), axis=0)
    assert np.all(np.abs(got["parts"] - ref["parts"]) <= 1e-9 * scale), \
        float(np.max(np.abs(got["parts"] - ref["parts"]) / scale))
    cs = np.max(np.abs(ref["C"]))
    assert np.max(np.abs(got["C"] - ref["C"])) <= 1e-9 * cs
    assert np.max(np.abs(got["S"] - ref["S"])) <= 1e-9 * np.max(np.abs(ref["S"]))
    assert abs(got["fwhm"] - ref["fwhm"]) <= 1e-9 * abs(ref["fwhm"]), (got["fwhm"], ref["fwhm"])
    assert abs(got["fwhm_se"] - ref["fwhm_se"]) <= 1e-7 * abs(ref["fwhm_se"]) + 1e-12
    assert abs(got["spsm_tau0"] - ref["C"][0].real) <= 1e-9 * cs
    # C(0+) is real up to O(eps) (the equal-time <S+S->)
    assert abs(got["C"][0].imag) <= 1e-2 * abs(got["C"][0].real)


@pytest.mark.parametrize("prec,route", [("bf16x3", "dense"), ("bf16x3", "fft"), ("fp32", "dense")])
def test_mixed_precision_within_standard_errors(prec, route):
    from paper_2608_10075_b300 import twa
    N, alpha, w, G, dt, seed = 64, 1.0, 16.0, 1.0, 2e-3, 8
    M, prep, lags, stride, eps, n_om, omax = 256, 200, 1000, 10, 1e-2, 321, 40.0
    ref = _reference(N, alpha, w, G, dt, seed, M, prep, lags, stride, eps, n_om, omax)
    with twa.TWA(N, alpha, w, G, dt, seed=seed, precision=prec, ws_route=route) as g:
        got = g.correlation(M, prep, lags, stride, eps, n_om, omax)
    # oracle standard errors of Re C and Im C per lag (same jackknife blocks)
    smp = ref["samples"]
    B = 32
    edges = [(b * M) // B for b in range(B + 1)]
    from oracle.two_time import correlation_from_parts
    tot = smp.sum(axis=1)
    est = np.stack([correlation_from_parts((tot - smp[:, edges[b]:edges[b + 1]].sum(axis=1)) /
                                           (M - (edges[b + 1] - edges[b]))) for b in range(B)])
    ref_se_re = np.sqrt((B - 1) / B * np.sum((est.real - est.real.mean(0)) ** 2, axis=0))
    ref_se_im = np.sqrt((B - 1) / B * np.sum((est.imag - est.imag.mean(0)) ** 2, axis=0))
    # (at lag 0 the imaginary part is exactly zero on both sides, with zero error)
    for part, g_, r_, se_ in (("re", got["C"].real, ref["C"].real, np.hypot(got["C_se"][:, 0], ref_se_re)),
                              ("im", got["C"].imag, ref["C"].imag, np.hypot(got["C_se"][:, 1], ref_se_im))):
        scale = np.max(np.abs(ref["C"]))
        assert np.all(np.abs(g_ - r_) <= 4.0 * se_ + 1e-9 * scale), (part, float(np.max(np.abs(g_ - r_) / (se_ + 1e-300))))
    assert abs(got["fwhm"] - ref["fwhm"]) <= 3.0 * math.hypot(got["fwhm_se"], ref["fwhm_se"]), \
        (got["fwhm"], ref["fwhm"], got["fwhm_se"], ref["fwhm_se"])


def test_correlation_rejects_bad_requests():
    from paper_2608_10075_b300 import twa
    with twa.TWA(16, 1.0, 4.0, 1.0, 1e-3, precision="fp64") as g:
        for args in ((8, 4, 4, 1, 0.0, 11, 5.0), (8, 4, 4, 0, 1e-3, 11, 5.0), (8, 4, 4, 1, 1e-3, 2, 5.0),
                     (0, 4, 4, 1, 1e-3, 11, 5.0), (8, 4, 4, 1, 1e-3, 11, -1.0)):
            with pytest.raises(twa.TWAError) as e:
                g.correlation(*args)
            assert e.value.name == "TWA_EINVAL", args
        # the context is untouched and still runs
        g.run(8, 3)
        g.sync()
