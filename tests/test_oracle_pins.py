"""Pins of the FP64 CPU oracle to things other than itself.

Each test checks the oracle against a value the paper, the mathematics or an
independent computation fixes: published Philox known-answer vectors, closed
forms of the TWA stationary laws, the spectrum asymptotics of the pump matrix,
an exact quantum solution for a few spins, and invariants of the equations of
motion. Chosen so that a dropped term, a flipped sign or a transposed operand
in the oracle fails at least one of them.
"""
import math
import os

import mpmath
import numpy as np
import pytest
import scipy.stats

from oracle import lindblad as lb
from oracle.twa_oracle import (TWAOracle, initial_signs, noise_factor, observables_from_moments,
                               philox4x32_10, philox_normals, pump_matrix, spectrum)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQRT3 = math.sqrt(3.0)


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(*r[:6])
        assert [int(v) for v in out] == r[6:]


def test_normals_are_standard_and_independent():
    m = np.arange(4096, dtype=np.uint64)[:, None]
    i = np.arange(50, dtype=np.uint64)[None, :]
    gx, gy = philox_normals(12345, m, np.uint64(7), i, 0)
    x, y = gx.ravel(), gy.ravel()
    n = x.size
    for v in (x, y):
        assert abs(v.mean()) < 5.0 / math.sqrt(n)
        assert abs(v.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
        assert scipy.stats.kstest(v, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(x, y)[0, 1]) < 5.0 / math.sqrt(n)
    # different steps and streams give uncorrelated draws
    hx, _ = philox_normals(12345, m, np.uint64(8), i, 0)
    assert abs(np.corrcoef(x, hx.ravel())[0, 1]) < 5.0 / math.sqrt(n)


def test_discrete_wigner_initial_state():
    m = np.arange(20000, dtype=np.uint64)[:, None]
    sx, sy = initial_signs(3, m, np.arange(4, dtype=np.uint64)[None, :])
    assert set(np.unique(sx)) == {-1.0, 1.0} and set(np.unique(sy)) == {-1.0, 1.0}
    n = sx.size
    # <sigma^x> = <sigma^y> = 0 and no correlation between components or sites
    assert abs(sx.mean()) < 5 / math.sqrt(n) and abs(sy.mean()) < 5 / math.sqrt(n)
    assert abs((sx * sy).mean()) < 5 / math.sqrt(n)
    assert abs((sx[:, 0] * sx[:, 1]).mean()) < 5 / math.sqrt(sx.shape[0])


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0, 3.0])
def test_wmin_matches_dirichlet_eta(alpha):
    # Below Eq. (3): w_min ~ w (2 eta(alpha) - 1), eta the Dirichlet eta function.
    _, wmin = spectrum(500, alpha, 2.5)
    target = 2.5 * (2.0 * float(mpmath.altzeta(alpha)) - 1.0)
    assert abs(wmin / target - 1.0) < 1e-4


@pytest.mark.parametrize("alpha,tol", [(2.0, 1e-2), (3.0, 1e-3)])
def test_wmax_short_range_limit(alpha, tol):
    # Eq. (3), alpha > 1: w_max is set by the zeta function; on the open chain the
    # bulk row sum is 1 + 2 (zeta(alpha) - 1) = 2 zeta(alpha) - 1.
    wmax, _ = spectrum(500, alpha, 1.0)
    assert abs(wmax / (2.0 * float(mpmath.zeta(alpha)) - 1.0) - 1.0) < tol


def test_wmax_long_range_scalings():
    # Eq. (3): w_max ~ w N^(1-alpha) for alpha < 1, ~ w log N at alpha = 1.
    a_small, _ = spectrum(250, 0.5, 1.0)
    a_big, _ = spectrum(1000, 0.5, 1.0)
    slope = math.log(a_big / a_small) / math.log(4.0)
    assert abs(slope - 0.5) < 0.05
    b_small, _ = spectrum(250, 1.0, 1.0)
    b_big, _ = spectrum(1000, 1.0, 1.0)
    # log growth: each factor 4 in N adds (2 ln 4) w up to O(1/N) terms
    assert abs((b_big - b_small) / (2.0 * math.log(4.0)) - 1.0) < 0.02


def test_pump_matrix_limits():
    W0 = pump_matrix(6, 0.0, 1.5)
    assert np.all(W0 == 1.5)                       # collective pump
    Winf = pump_matrix(6, math.inf, 1.5)
    assert np.array_equal(Winf, 1.5 * np.eye(6))    # local pump
    W = pump_matrix(5, 1.0, 2.0)
    assert W[0, 0] == 2.0 and W[0, 1] == 1.0 and W[4, 0] == 2.0 / 5.0 and W[1, 3] == 2.0 / 3.0


def test_pump_matrix_rounding_breaks_definiteness_near_alpha_zero():
    # Eq. 2 is positive definite for every alpha > 0 (convex decreasing sequence),
    # but at alpha = 1e-15 the entries differ from w by a few ulps only, so the
    # stored FP64 matrix is rank one plus rounding noise of both signs: it has a
    # negative eigenvalue and no Cholesky factor. This is the case the clip
    # option of the library is tested on; at alpha = 1e-12 the spread
    # alpha ln(1 + |i-j|) is far above the rounding and the factor exists.
    N, w = 200, 5.0
    W = pump_matrix(N, 1e-15, w)
    assert np.linalg.eigvalsh(W)[0] < 0.0
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(W)
    W12 = pump_matrix(N, 1e-12, w)
    assert np.linalg.eigvalsh(W12)[0] > 0.0
    np.linalg.cholesky(W12)


@pytest.mark.parametrize("alpha", [0.0, 0.75, 2.0, math.inf])
def test_noise_covariance_equals_pump_times_dt(alpha):
    # Sec. S1: <chi_i chi_j> = w_ij delta(t-t'), <xi xi> = Gamma delta(t-t').
    N, M, dt, G, w = 6, 40000, 0.01, 1.3, 2.0
    o = TWAOracle(N, alpha, w, G, dt, 99, M)
    dxi_x, dxi_y, dchi_x, dchi_y = o.noise_increments(5)
    W = pump_matrix(N, alpha, w)
    for dchi in (dchi_x, dchi_y):
        C = dchi.T @ dchi / M
        tol = 6.0 * w * dt * math.sqrt(2.0 / M)
        assert np.max(np.abs(C - W * dt)) < tol
    assert abs(np.mean(dchi_x * dchi_y)) < 6.0 * w * dt / math.sqrt(M)
    for dxi in (dxi_x, dxi_y):
        assert abs(np.mean(dxi ** 2) / (G * dt) - 1.0) < 6.0 * math.sqrt(2.0 / M)
        assert dxi.shape == (M, 1)          # one collective noise per trajectory
    assert abs(np.mean(dxi_x * dxi_y)) < 6.0 * G * dt / math.sqrt(M)


def test_increment_is_a_rotation():
    # Sec. S1: ds_i = s_i x b_i, so s_i . ds_i = 0 for any state and any noise.
    rng = np.random.default_rng(0)
    N, M = 7, 16
    o = TWAOracle(N, 0.8, 3.0, 1.7, 0.01, 5, M)
    sx, sy, sz = (rng.normal(size=(M, N)) for _ in range(3))
    dxi_x, dxi_y, dchi_x, dchi_y = o.noise_increments(3)
    dx, dy, dz = o.increment(sx, sy, sz, dxi_x, dxi_y, dchi_x, dchi_y)
    dot = sx * dx + sy * dy + sz * dz
    assert np.max(np.abs(dot)) < 1e-12 * np.max(np.abs(dx) + np.abs(dy) + np.abs(dz))
    # and the noise enters through s^z for the transverse components (Eq. (S1))
    dx0, dy0, dz0 = o.increment(sx, sy, np.zeros_like(sz), dxi_x, dxi_y, dchi_x, dchi_y)
    assert np.all(dx0 == 0.0) and np.all(dy0 == 0.0)


def _single_spin_sz(dt, M, seed):
    o = TWAOracle(1, 1.0, 8.0, 1.0, dt, seed, M, init_sz=-1.0, window_start=2.0)
    o.run(int(round(12.0 / dt)))
    ob = o.observables()
    return ob["Sz"], ob["Sz_se"]


def test_single_spin_stationary_law():
    # N = 1: collective decay = local decay. Stratonovich Fokker-Planck on the
    # sphere |s| = sqrt(3) gives p(s^z) ~ exp(-a s^z) with a = (Gamma-w)/(Gamma+w),
    # so <s^z> = 1/a - sqrt(3) coth(sqrt(3) a). Heun is weak order 1, so the
    # Richardson combination 2 f(dt) - f(2 dt) removes the O(dt) bias.
    w, G = 8.0, 1.0
    a = (G - w) / (G + w)
    exact = 1.0 / a - SQRT3 / math.tanh(SQRT3 * a)
    f1, s1 = _single_spin_sz(0.004, 8192, 11)
    f2, s2 = _single_spin_sz(0.008, 8192, 12)
    extrap = 2.0 * f1 - f2
    se = math.sqrt(4.0 * s1 * s1 + s2 * s2)
    assert abs(extrap - exact) < 3.5 * se
    # the raw estimates approach the law from one side as dt shrinks
    assert abs(f1 - exact) < abs(f2 - exact) + 3.0 * math.hypot(s1, s2)


def test_collective_pump_uniform_sphere():
    # alpha = 0, w = Gamma: every spin sees the same field, the total spin S
    # rotates rigidly with no drift, so S is uniform on its sphere |S| = R.
    # With R^2 = (S^x)^2 + (S^y)^2 + N^2 from the +-1 initial signs:
    # <S^z> = 0, <(S^z)^2> = <R^2>/3, <A> = <R^2>/6, <A^2> = <R^4>/30.
    N, M = 8, 3072
    o = TWAOracle(N, 0.0, 1.0, 1.0, 0.005, 21, M, init_sz=-1.0, window_start=3.0)
    o.run(2000)
    mu = o.window_means()
    se = mu.std(axis=0, ddof=1) / math.sqrt(M)
    R2 = N * N + 2.0 * N
    R4 = N ** 4 + 4.0 * N ** 3 + 8.0 * N * N - 4.0 * N
    target = {0: 0.0, 1: R2 / 6.0, 2: R4 / 30.0, 4: R2 / 3.0}
    for k, v in target.items():
        assert abs(mu[:, k].mean() - v) < 4.0 * se[k] + 0.01 * abs(v), (k, mu[:, k].mean(), v, se[k])


def test_spin_length_heun_drift_order():
    # Every term of Eq. (S1) is a rotation, so |s_i|^2 = 3 is conserved by the
    # continuous dynamics. Without renormalisation the Stratonovich-Heun step
    # drifts by O(dt^2) per step; an Ito/Euler step would drift by O(dt).
    drift = []
    for dt in (1e-2, 2.5e-3):
        o = TWAOracle(8, 1.0, 4.0, 1.0, dt, 3, 512, init_sz=-1.0, renormalize=False)
        o.run(1)
        drift.append(np.mean(np.abs(o.sx ** 2 + o.sy ** 2 + o.sz ** 2 - 3.0)))
    assert drift[0] / drift[1] > 12.0
    o = TWAOracle(8, 1.0, 4.0, 1.0, 1e-2, 3, 64, init_sz=-1.0, renormalize=True)
    o.run(5)
    assert np.max(np.abs(o.sx ** 2 + o.sy ** 2 + o.sz ** 2 - 3.0)) < 1e-13


def test_brute_force_matches_dicke_closed_form():
    # Sec. S3: collective pump and decay, detailed balance p_{m+1} = (w/Gamma) p_m
    # inside J = N/2; g2 -> 6/5 at w = Gamma for large N.
    N = 4
    for w in (0.5, 1.0, 3.0):
        rho = lb.steady_state(N, pump_matrix(N, 0.0, w), 1.0, T=400.0)
        ex = lb.expectations(rho, N)
        cf = lb.dicke_collective_steady(N, w, 1.0)
        for k in ("Sz", "SpSm", "G2num"):
            assert abs(ex[k] - cf[k]) < 1e-8 * max(1.0, abs(cf[k]))
    assert abs(lb.dicke_collective_steady(4000, 1.0, 1.0)["g2"] - 1.2) < 1e-3


def test_twa_close_to_exact_at_weak_pump():
    # Weak pump (normalised pump w_max / (Gamma N) ~ 0.27 here): the paper reports
    # quantitative agreement of TWA with the exact solution in this regime. TWA
    # first moments are not exact, so the tolerance is the observed TWA error
    # (about 3 %) with margin, not a standard error.
    N, alpha, w = 4, 1.0, 0.5
    ex = lb.expectations(lb.steady_state(N, pump_matrix(N, alpha, w), 1.0, T=200.0), N)
    o = TWAOracle(N, alpha, w, 1.0, 0.01, 17, 2048, init_sz=-1.0, window_start=20.0)
    o.run(6000)
    ob = o.observables()
    assert abs(ob["Sz"] - ex["Sz"]) < 0.08 * abs(ex["Sz"]) + 3 * ob["Sz_se"]
    assert abs(ob["SpSm"] - ex["SpSm"]) < 0.05 * abs(ex["SpSm"]) + 3 * ob["SpSm_se"]
    # a flipped pump sign would drive the chain to S^z = -N instead
    assert ob["Sz"] > -0.5 * N


@pytest.mark.parametrize("alpha", [0.5, 2.0])
def test_direct_steady_state_equals_time_evolution(alpha):
    # the reduced direct solve (popcount sector, real symmetric unknowns) against
    # the long-time limit of the full dense superoperator, a method with neither
    # reduction; and the sparse superoperator equals the dense one term for term
    N, w = 4, 0.7
    W = pump_matrix(N, alpha, w)
    assert np.array_equal(lb.liouvillian_sparse(N, W, 1.0).toarray(), lb.liouvillian(N, W, 1.0))
    a = lb.steady_state_unique(N, W, 1.0)
    b = lb.steady_state(N, W, 1.0, T=400.0)
    assert np.max(np.abs(a - b)) < 1e-10
    with pytest.raises(ValueError):
        lb.steady_state_unique(N, pump_matrix(N, 0.0, w), 1.0)   # collective pump: not unique


def test_direct_steady_state_n8_is_a_stationary_density_matrix():
    N = 8
    W = pump_matrix(N, 1.0, 0.5)
    rho = lb.steady_state_unique(N, W, 1.0)
    L = lb.liouvillian_sparse(N, W, 1.0)
    res = L @ rho.reshape(-1, order="F")
    assert np.max(np.abs(res)) < 1e-12 * abs(L).max()
    assert abs(np.trace(rho) - 1.0) < 1e-12
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    ex = lb.expectations(rho, N)
    # between the empty state (S^z = -N) and the normalised pump's weak-pump regime
    assert -N < ex["Sz"] < 0.0 and ex["SpSm"] > 0.0


def test_twa_close_to_exact_at_weak_pump_n8():
    # N = 8 (the largest brute-force case): TWA against the exact steady state in
    # the weak-pump regime; observed TWA errors 2.3 % (S^z), 0.6 % (<S+S->), 2.7 %
    # (g2) with 2048 trajectories, so the tolerances leave a margin, not a
    # standard-error bound
    N, alpha, w = 8, 1.0, 0.5
    ex = lb.expectations(lb.steady_state_unique(N, pump_matrix(N, alpha, w), 1.0), N)
    o = TWAOracle(N, alpha, w, 1.0, 0.01, 23, 1024, init_sz=-1.0, window_start=20.0)
    o.run(6000)
    ob = o.observables()
    assert abs(ob["Sz"] - ex["Sz"]) < 0.06 * abs(ex["Sz"]) + 3 * ob["Sz_se"]
    assert abs(ob["SpSm"] - ex["SpSm"]) < 0.03 * abs(ex["SpSm"]) + 3 * ob["SpSm_se"]
    assert abs(ob["g2"] - ex["g2"]) < 0.05 * abs(ex["g2"]) + 3 * ob["g2_se"]


def test_special_cases():
    # No decay and no pump: the state never moves.
    o = TWAOracle(5, 1.0, 0.0, 0.0, 0.01, 2, 16, init_sz=-1.0)
    x0, y0, z0 = o.sx.copy(), o.sy.copy(), o.sz.copy()
    o.run(10)
    assert np.array_equal(o.sx, x0) and np.array_equal(o.sy, y0) and np.array_equal(o.sz, z0)
    # Local pump (alpha = inf) without decay: independent spins, each with the
    # single-spin law at a = -1: <sigma^z> = -1 + sqrt(3) coth(sqrt(3)).
    o = TWAOracle(4, math.inf, 2.0, 0.0, 0.004, 4, 2048, init_sz=-1.0, window_start=3.0)
    o.run(2000)
    ob = o.observables()
    exact = -1.0 + SQRT3 / math.tanh(SQRT3)
    assert abs(ob["sigma_z"] - exact) < 4.0 * ob["sigma_z_se"] + 0.02


@pytest.mark.parametrize("init_sz", [-1.0, 1.0])
def test_normal_ordering_on_product_states(init_sz):
    # Sec. S1, item 6, applied to the discrete-Wigner samples of a product state
    # at t = 0. All down: <S+S-> = 0 exactly and the four-point estimator gives
    # -7N/12; all up: <S+S-> = N and the estimator gives 2N^2 - 5N/4. These are
    # closed-form expectations over the +-1 samples (moments 1, N, 3N^2 - 2N).
    N, M = 6, 200000
    m = np.arange(M, dtype=np.uint64)[:, None]
    sx, sy = initial_signs(8, m, np.arange(N, dtype=np.uint64)[None, :])
    Sx, Sy, Sz = sx.sum(1), sy.sum(1), np.full(M, init_sz * N)
    A = 0.25 * (Sx * Sx + Sy * Sy)
    ob = observables_from_moments(np.stack([Sz, A, A * A, A * Sz, Sz * Sz], axis=1), N)
    if init_sz < 0:
        spsm, g2n = 0.0, -7.0 * N / 12.0
    else:
        spsm, g2n = float(N), 2.0 * N * N - 1.25 * N
    assert abs(ob["SpSm"] - spsm) < 4 * ob["SpSm_se"] + 1e-12
    assert abs(ob["G2num"] - g2n) < 4 * ob["G2num_se"]


def test_continuation_is_exact():
    # Counter-based noise: 7 + 5 steps reproduce 12 steps bit for bit.
    a = TWAOracle(6, 1.0, 3.0, 1.0, 0.01, 5, 32, window_start=0.0)
    a.run(12)
    b = TWAOracle(6, 1.0, 3.0, 1.0, 0.01, 5, 32, window_start=0.0)
    b.run(7)
    b.run(5)
    assert np.array_equal(a.sx, b.sx) and np.array_equal(a.sz, b.sz)
    assert np.array_equal(a.mom, b.mom)
    # a trajectory subset (m0 offset) reproduces the same rows of the full run
    c = TWAOracle(6, 1.0, 3.0, 1.0, 0.01, 5, 8, m0=10, window_start=0.0)
    c.run(12)
    assert np.array_equal(c.sx, a.sx[10:18])


def test_g2_jackknife_on_known_law():
    # Ratio estimator on samples with a known answer: independent Gaussian
    # moments; the jackknife SE should match the spread over repetitions.
    rng = np.random.default_rng(4)
    vals = []
    ses = []
    for _ in range(60):
        M = 512
        s = np.column_stack([rng.normal(0, 1, M), rng.normal(10, 1, M), rng.normal(130, 5, M),
                             rng.normal(0, 1, M), rng.normal(5, 1, M)])
        ob = observables_from_moments(s, 4)
        vals.append(ob["g2"])
        ses.append(ob["g2_se"])
    spread = np.std(vals, ddof=1)
    assert 0.7 < np.mean(ses) / spread < 1.4
    # g2 = (130 + 0 - 0 + 2.5 - 40/3) / 10^2 for these means
    assert abs(np.mean(vals) - (130 + 2.5 - 40.0 / 3.0) / 100.0) < 4 * spread / math.sqrt(60)


def test_sample_stride_takes_every_kth_step_of_the_window():
    # Same trajectories (same seed and counters): with stride k the window mean is
    # the mean of the states after steps n_w + k, n_w + 2k, ... <= T.
    N, M, steps, nw, k, dt = 5, 7, 23, 4, 3, 0.01
    states = {}

    class Record(TWAOracle):
        def step(self):
            super().step()
            states[self.t] = (self.sx.sum(1), self.sy.sum(1), self.sz.sum(1))

    a = Record(N, 1.0, 3.0, 1.0, dt, 9, M, window_start=nw * dt)
    a.run(steps)
    b = TWAOracle(N, 1.0, 3.0, 1.0, dt, 9, M, window_start=nw * dt, sample_stride=k)
    b.run(steps)
    picks = [t for t in sorted(states) if t > nw and (t - nw) % k == 0]
    assert picks == list(range(nw + k, steps + 1, k)) and b.count == len(picks)
    assert np.array_equal(a.sx, b.sx)
    Sz = np.mean([states[t][2] for t in picks], axis=0)
    A = np.mean([0.25 * (states[t][0] ** 2 + states[t][1] ** 2) for t in picks], axis=0)
    assert np.allclose(b.window_means()[:, 0], Sz, rtol=1e-13, atol=1e-12)
    assert np.allclose(b.window_means()[:, 1], A, rtol=1e-13, atol=1e-12)
    # stride 1 is every step of the window
    assert a.count == steps - nw
