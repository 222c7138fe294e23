"""Pins of the oracle's FP64 tangent (pathwise derivatives at fixed noise).

The tangent is checked against central finite differences of the oracle's
forward integrator with common random numbers: the same seed and counters
give the same noise draws at theta +- delta, so the difference quotient is the
same pathwise derivative up to O(delta^2). The Cholesky derivative is checked
against differences of the library Cholesky factorisation.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import noise_factor
from oracle.twa_tangent import (TWATangent, factor_derivative, finite_difference, objective_coefficients,
                                pump_derivative)


@pytest.mark.parametrize("alpha", [0.4, 1.1, 2.5])
@pytest.mark.parametrize("theta", ["w", "alpha"])
def test_cholesky_derivative_matches_differences(alpha, theta):
    N, w, d = 14, 3.0, 1e-6
    L = noise_factor(N, alpha, w)
    dL = factor_derivative(L, pump_derivative(N, alpha, w, theta), alpha, w)
    if theta == "w":
        fd = (noise_factor(N, alpha, w * (1 + d)) - noise_factor(N, alpha, w * (1 - d))) / (2 * w * d)
    else:
        fd = (noise_factor(N, alpha + d, w) - noise_factor(N, alpha - d, w)) / (2 * d)
    assert np.max(np.abs(dL - fd)) < 1e-8 * max(1.0, np.max(np.abs(dL)))
    # and L dL^T + dL L^T = dW (derivative of L L^T = W)
    dW = pump_derivative(N, alpha, w, theta)
    assert np.max(np.abs(L @ dL.T + dL @ L.T - dW)) < 1e-11 * np.max(np.abs(dW))


@pytest.mark.parametrize("objective", ["SpSm", "g2"])
@pytest.mark.parametrize("theta", ["w", "alpha"])
@pytest.mark.parametrize("alpha", [1.0, 0.3])
def test_tangent_matches_crn_finite_difference(objective, theta, alpha):
    N, w, G, dt, M, steps = 12, 8.0, 1.0, 2e-3, 48, 50
    kw = dict(window_start=0.04)
    o = TWATangent(N, alpha, w, G, dt, 3, M, theta, **kw)
    o.run(steps)
    J, dJ, per = o.derivative(objective)
    fd = finite_difference(N, alpha, w, G, dt, 3, M, steps, theta, objective, 1e-5, **kw)
    assert abs(dJ - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(J)), (dJ, fd)
    assert per.shape == (M,) and abs(per.mean() - dJ) < 1e-14 * max(1.0, abs(dJ))


@pytest.mark.parametrize("alpha", [0.0, math.inf])
def test_tangent_special_factors(alpha):
    # closed-form factors: rank one (alpha = 0) and diagonal (alpha = inf), d/dw only
    N, w, G, dt, M, steps = 10, 2.0, 1.0, 2e-3, 32, 40
    o = TWATangent(N, alpha, w, G, dt, 1, M, "w")
    o.run(steps)
    J, dJ, _ = o.derivative("SpSm")
    fd = finite_difference(N, alpha, w, G, dt, 1, M, steps, "w", "SpSm", 1e-5)
    assert abs(dJ - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(J))


def test_objective_coefficients_are_the_gradient_of_the_estimators():
    # c for g2 is the gradient of g2num / spsm^2 w.r.t. the five means (numerical check)
    mu = np.array([3.0, 10.0, 130.0, 20.0, 12.0])
    for obj in ("SpSm", "g2"):
        c, J = objective_coefficients(mu, obj)
        for k in range(5):
            e = np.zeros(5)
            e[k] = 1e-6 * max(1.0, abs(mu[k]))
            d = (objective_coefficients(mu + e, obj)[1] - objective_coefficients(mu - e, obj)[1]) / (2 * e[k])
            assert abs(d - c[k]) < 1e-7 * max(1.0, abs(c[k]))
