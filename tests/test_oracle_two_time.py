"""Pins of the two-time oracle (oracle/two_time.py), each against something
other than itself: single-spin quantum mechanics for the kick, the equal-time
estimator of Sec. S1 item 6 at tau -> 0+, the closed-form deterministic flow
of one decaying spin for the responses, the eps -> 0 limit for the shared
noise of the copies, and an analytic Lorentzian for the spectrum and width.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle, observables_from_moments
from oracle.two_time import correlation_from_parts, fwhm, kick, spectrum, two_time, two_time_samples

PAULI = {"x": np.array([[0, 1], [1, 0]], dtype=complex), "y": np.array([[0, -1j], [1j, 0]]),
         "z": np.array([[1, 0], [0, -1]], dtype=complex)}


@pytest.mark.parametrize("axis", ["x", "y"])
def test_kick_is_the_unitary_of_eps_sigma(axis):
    # rho' = U rho U^+ with U = exp(-i eps sigma^axis): the Bloch vector of rho'
    # is the classical kick of the Bloch vector of rho (the map is linear in s,
    # so any length works)
    eps = 0.137
    rng = np.random.default_rng(1)
    for _ in range(5):
        s = rng.normal(size=3)
        s *= 0.9 / np.linalg.norm(s)
        rho = 0.5 * (np.eye(2) + sum(s[k] * PAULI[a] for k, a in enumerate("xyz")))
        U = math.cos(eps) * np.eye(2) - 1j * math.sin(eps) * PAULI[axis]
        r2 = U @ rho @ U.conj().T
        expect = np.array([np.trace(r2 @ PAULI[a]).real for a in "xyz"])
        got = np.array(kick(np.array([s[0]]), np.array([s[1]]), np.array([s[2]]), axis, eps)).ravel()
        assert np.allclose(got, expect, atol=1e-13), (axis, got, expect)


def test_equal_time_limit_is_the_normal_ordered_estimator():
    # lag 0 (right after the kick): <S+(0+) S-(0)> = A + <S^z>/2 (Sec. S1 item 6)
    # up to O(eps); the imaginary part vanishes
    N, M, eps = 24, 64, 1e-6
    smp = two_time_samples(N, 1.0, 6.0, 1.0, 1e-3, 3, M, 40, 0, 1, eps)
    C0 = correlation_from_parts(smp[0].mean(axis=0))
    o = TWAOracle(N, 1.0, 6.0, 1.0, 1e-3, 3, M)
    o.run(40)
    Sx, Sy, Sz = o.sx.sum(1), o.sy.sum(1), o.sz.sum(1)
    ref = np.mean(0.25 * (Sx * Sx + Sy * Sy) + 0.5 * Sz)
    assert abs(C0.real - ref) <= 1e-4 * N, (C0, ref)
    assert abs(C0.imag) <= 1e-4 * N
    # and it is the observable the equal-time reduction reports for that state
    mom = np.stack([Sz, 0.25 * (Sx * Sx + Sy * Sy), 0 * Sz, 0 * Sz, Sz * Sz], axis=1)
    assert abs(observables_from_moments(mom, N)["SpSm"] - ref) < 1e-9 * abs(ref)


class _NoNoise(TWAOracle):
    """The oracle's integrator with every noise term set to zero."""

    def noise(self, t):
        xi_x, xi_y, eta_x, eta_y = super().noise(t)
        return 0 * xi_x, 0 * xi_y, 0 * eta_x, 0 * eta_y


def _decay_flow(s, Gamma, t):
    """Closed form of one spin under collective decay alone (N = 1, no noise):
    dz/dt = -Gamma/2 (3 - z^2) on |s| = sqrt 3 gives z = -sqrt3 tanh(u0 + sqrt3 Gamma t / 2),
    u0 = atanh(-z0 / sqrt3); the transverse part shrinks by cosh(u0) / cosh(u)."""
    x0, y0, z0 = s
    u0 = math.atanh(-z0 / math.sqrt(3.0))
    u = u0 + 0.5 * math.sqrt(3.0) * Gamma * t
    f = math.cosh(u0) / math.cosh(u)
    return np.array([x0 * f, y0 * f, -math.sqrt(3.0) * math.tanh(u)])


def test_responses_follow_the_closed_form_flow():
    # N = 1, Gamma = 1, w = 0, noise off: the two-time quantities of the oracle
    # against the closed-form flow from the kicked states (responses by a
    # central difference of the closed form, which is smooth in eps)
    G, dt, prep, lags, stride, eps = 1.0, 1e-3, 200, 600, 100, 1e-5
    smp = two_time_samples(1, 1.0, 0.0, G, dt, 5, 4, prep, lags, stride, eps, oracle_cls=_NoNoise)
    o = _NoNoise(1, 1.0, 0.0, G, dt, 5, 4)
    o.run(prep)
    for m in range(4):
        s0 = np.array([o.sx[m, 0], o.sy[m, 0], o.sz[m, 0]])
        for k in range(smp.shape[0]):
            tau = k * stride * dt
            sa = _decay_flow(s0, G, tau)
            h = 1e-4
            resp = {}
            for axis in ("x", "y"):
                sp = _decay_flow(np.array(kick(*(np.array([v]) for v in s0), axis, h)).ravel(), G, tau)
                sm = _decay_flow(np.array(kick(*(np.array([v]) for v in s0), axis, -h)).ravel(), G, tau)
                resp[axis] = (sp - sm) / (2 * h)
            ref = [sa[0] * s0[0], sa[1] * s0[1], sa[0] * s0[1], sa[1] * s0[0],
                   resp["x"][0], resp["x"][1], resp["y"][0], resp["y"][1]]
            # Heun's O(dt^2) global error and the O(eps) of the one-sided difference
            assert np.allclose(smp[k, m], ref, rtol=1e-4, atol=1e-4), (m, k, smp[k, m], ref)


def test_copies_share_their_noise():
    # with the noise on, the responses converge as eps -> 0 only if the copies
    # see the same noise (a copy with other noise would differ by O(1) / eps)
    a = two_time_samples(6, 1.0, 4.0, 1.0, 2e-3, 9, 8, 20, 30, 10, 1e-5)
    b = two_time_samples(6, 1.0, 4.0, 1.0, 2e-3, 9, 8, 20, 30, 10, 1e-6)
    assert np.allclose(a[..., 4:], b[..., 4:], rtol=1e-3, atol=1e-3)
    assert np.array_equal(a[..., :4], b[..., :4])   # the unperturbed copy does not see eps


def test_spectrum_and_width_of_a_lorentzian():
    # C(tau) = C0 exp(-gamma tau / 2 - i w0 tau): S(omega) = 2 C0 (gamma/2) / ((gamma/2)^2 + (omega - w0)^2),
    # FWHM = gamma, peak at w0
    # (a coarse lag grid, so that the trapezoid end weights matter at 1e-2)
    C0, gamma, w0, dtau = 7.0, 0.8, 0.3, 0.05
    tau = np.arange(0, 60.0, dtau)
    C = C0 * np.exp(-0.5 * gamma * tau - 1j * w0 * tau)
    om = np.linspace(-3, 3, 1201)
    S = spectrum(C, dtau, om)
    ref = 2 * C0 * (0.5 * gamma) / ((0.5 * gamma) ** 2 + (om - w0) ** 2)
    assert np.max(np.abs(S - ref)) <= 1e-3 * np.max(ref)
    assert abs(fwhm(om, S) - gamma) <= 2e-3 * gamma
    assert abs(om[np.argmax(S)] - w0) <= om[1] - om[0]
    assert math.isnan(fwhm(om, np.ones_like(om)))   # no half-maximum crossing


def test_static_spins_keep_their_correlation():
    # Gamma = w = 0: nothing moves, so every recorded lag repeats lag 0
    out = two_time(5, 1.0, 0.0, 0.0, 1e-3, 2, 16, 3, 40, 10, 1e-4, np.linspace(-1, 1, 21), blocks=4)
    assert out["parts"].shape == (5, 8)
    assert np.allclose(out["parts"], out["parts"][0], rtol=0, atol=1e-9)


def test_classical_part_is_the_product_of_complex_collective_spins():
    # a rigid rotation of the collective spin about z at rate w0: X = S^x + i S^y
    # goes to X e^{i w0 t}, so 1/4 <X(t) X(0)*> = |X0|^2 e^{i w0 t} / 4; the eight
    # quantities of those states must give exactly that (responses zero)
    rng = np.random.default_rng(2)
    X0 = rng.normal(size=50) + 1j * rng.normal(size=50)
    for t in (0.0, 0.7, 2.3):
        Xt = X0 * np.exp(1j * 0.9 * t)
        p = np.stack([Xt.real * X0.real, Xt.imag * X0.imag, Xt.real * X0.imag, Xt.imag * X0.real,
                      0 * X0.real, 0 * X0.real, 0 * X0.real, 0 * X0.real], axis=1).mean(axis=0)
        ref = np.mean(0.25 * Xt * np.conj(X0))
        assert abs(correlation_from_parts(p) - ref) <= 1e-12 * abs(ref), (t, correlation_from_parts(p), ref)
