"""Pins of the oracle's semi-implicit midpoint integrator (CPU).

The scheme the paper cites for its own runs (Mentink et al. 2010) takes each
stage as an implicit-midpoint rotation s' = s + ((s + s')/2) x b. These tests
check it against facts fixed outside the oracle: the rotation it must be
(Rodrigues' formula with angle 2 atan(|b|/2)), exact conservation of |s_i|,
consistency with the Heun step (the two differ by O(dt^{3/2}) per step while
the increment is O(dt^{1/2})), and the closed-form single-spin stationary law
of the Stratonovich dynamics.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import TWAOracle, pump_matrix

SQRT3 = math.sqrt(3.0)


def test_cayley_step_is_the_rodrigues_rotation():
    # ds = s x b = -b x s: a rotation about b / |b| by -2 atan(|b| / 2)
    rng = np.random.default_rng(1)
    s = rng.normal(size=(200, 3))
    b = rng.normal(size=(200, 3)) * rng.uniform(0.01, 3.0, size=(200, 1))
    out = np.stack(TWAOracle.cayley(s[:, 0], s[:, 1], s[:, 2], b[:, 0], b[:, 1], b[:, 2]), axis=-1)
    nb = np.linalg.norm(b, axis=1, keepdims=True)
    n = b / nb
    phi = -2.0 * np.arctan(nb / 2.0)
    rod = s * np.cos(phi) + np.cross(n, s) * np.sin(phi) + n * np.sum(n * s, axis=1, keepdims=True) * (1 - np.cos(phi))
    assert np.max(np.abs(out - rod)) < 1e-13 * np.max(np.abs(s))
    # and it solves the implicit equation it is defined by
    assert np.max(np.abs(out - s - np.cross(0.5 * (s + out), b))) < 1e-13 * np.max(np.abs(s))


def test_midpoint_keeps_every_spin_length_without_renormalisation():
    # each stage is an exact rotation, so |s_i|^2 = 3 to rounding after many
    # steps, where Heun without renormalisation drifts
    o = TWAOracle(8, 1.0, 4.0, 1.0, 1e-2, 3, 64, integrator="midpoint", renormalize=False)
    o.run(300)
    assert np.max(np.abs(o.sx ** 2 + o.sy ** 2 + o.sz ** 2 - 3.0)) < 1e-12
    h = TWAOracle(8, 1.0, 4.0, 1.0, 1e-2, 3, 64, integrator="heun", renormalize=False)
    h.run(300)
    assert np.max(np.abs(h.sx ** 2 + h.sy ** 2 + h.sz ** 2 - 3.0)) > 1e-4


def test_midpoint_and_heun_steps_agree_to_higher_order():
    # from the same state with the same noise: increments ~ dt^{1/2}, the
    # difference of the two schemes ~ dt^{3/2} (both Stratonovich-consistent)
    diff, inc = [], []
    for dt in (1e-2, 1e-2 / 16):
        st = {}
        for integ in ("heun", "midpoint"):
            o = TWAOracle(6, 1.0, 4.0, 1.0, dt, 3, 256, integrator=integ, renormalize=False)
            o.run(1)
            st[integ] = np.stack([o.sx, o.sy, o.sz])
        o0 = TWAOracle(6, 1.0, 4.0, 1.0, dt, 3, 256)
        s0 = np.stack([o0.sx, o0.sy, o0.sz])
        diff.append(np.abs(st["heun"] - st["midpoint"]).mean())
        inc.append(np.abs(st["heun"] - s0).mean())
    assert 2.5 < inc[0] / inc[1] < 6.5          # 16^{1/2} = 4
    assert diff[0] / diff[1] > 32.0             # 16^{3/2} = 64


def test_midpoint_is_second_order_without_noise():
    # With the noises switched off Eq. (S1) is the ODE ds_i/dt = s_i x b_i(s). The
    # scheme is the implicit midpoint rule with its field taken at the midpoint of
    # s and the predictor, which is second order; a field taken at the predictor
    # (or at s) would make it first order. Reference: RK4 at dt = 1e-4 of the rate
    # written out here from Eq. (S1) and the pump matrix.
    N, alpha, w, G, T, M = 5, 1.0, 3.0, 1.0, 0.5, 6
    W = pump_matrix(N, alpha, w)

    def rate(s):
        sx, sy, sz = s
        Bx = 0.5 * (G * sx.sum(1, keepdims=True) - sx @ W.T)
        By = 0.5 * (G * sy.sum(1, keepdims=True) - sy @ W.T)
        return np.stack([sz * Bx, sz * By, -(sx * Bx + sy * By)])

    o0 = TWAOracle(N, alpha, w, G, 0.1, 4, M)
    ref = np.stack([o0.sx, o0.sy, o0.sz])
    h = 1e-4
    for _ in range(int(round(T / h))):
        k1 = rate(ref)
        k2 = rate(ref + 0.5 * h * k1)
        k3 = rate(ref + 0.5 * h * k2)
        k4 = rate(ref + h * k3)
        ref = ref + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    err = []
    for dt in (0.05, 0.025, 0.0125):
        o = TWAOracle(N, alpha, w, G, dt, 4, M, renormalize=False, integrator="midpoint")
        z1, zN = np.zeros((M, 1)), np.zeros((M, N))
        o.noise_increments = lambda t: (z1, z1, zN, zN)
        o.run(int(round(T / dt)))
        err.append(np.max(np.abs(np.stack([o.sx, o.sy, o.sz]) - ref)))
    assert 3.5 < err[0] / err[1] < 4.5 and 3.5 < err[1] / err[2] < 4.5, err


def _single_spin_sz(dt, M, seed):
    o = TWAOracle(1, 1.0, 8.0, 1.0, dt, seed, M, init_sz=-1.0, window_start=2.0, integrator="midpoint")
    o.run(int(round(12.0 / dt)))
    ob = o.observables()
    return ob["Sz"], ob["Sz_se"]


def test_midpoint_single_spin_stationary_law():
    # N = 1: p(s^z) ~ exp(-a s^z) on the sphere |s| = sqrt(3), a = (G - w)/(G + w),
    # <s^z> = 1/a - sqrt(3) coth(sqrt(3) a) for the Stratonovich dynamics; the
    # scheme converges at weak order 1, so 2 f(dt) - f(2 dt) removes the bias.
    w, G = 8.0, 1.0
    a = (G - w) / (G + w)
    exact = 1.0 / a - SQRT3 / math.tanh(SQRT3 * a)
    f1, s1 = _single_spin_sz(0.004, 8192, 31)
    f2, s2 = _single_spin_sz(0.008, 8192, 32)
    extrap = 2.0 * f1 - f2
    se = math.sqrt(4.0 * s1 * s1 + s2 * s2)
    assert abs(extrap - exact) < 3.5 * se, (f1, f2, extrap, exact, se)


def test_midpoint_collective_pump_uniform_sphere():
    # alpha = 0, w = Gamma: the total spin rotates rigidly with no drift, so it is
    # uniform on its sphere |S| = R: <S^z> = 0 and <(S^z)^2> = <R^2>/3 with
    # <R^2> = N^2 + 2N for the +-1 initial signs
    N, M = 8, 1024
    o = TWAOracle(N, 0.0, 1.0, 1.0, 0.005, 21, M, init_sz=-1.0, window_start=3.0, integrator="midpoint")
    o.run(1400)
    mu = o.window_means()
    se = mu.std(axis=0, ddof=1) / math.sqrt(M)
    assert abs(mu[:, 0].mean()) < 4.0 * se[0]
    assert abs(mu[:, 4].mean() - (N * N + 2.0 * N) / 3.0) < 4.0 * se[4]


def test_integrator_name_is_checked():
    with pytest.raises(ValueError):
        TWAOracle(2, 1.0, 1.0, 1.0, 0.1, 0, 2, integrator="euler")
