"""FP64 forward-mode tangent of the TWA oracle: pathwise derivatives at fixed noise.

TEST INFRASTRUCTURE (same rules as twa_oracle.py: only tests/, smoke() and the
CPU leg of bench.py use it; the product library never does).

For a parameter theta in {w, alpha} of the pump matrix (Eq. 2), the noise draws
(eta, xi) are held fixed and every quantity of one stochastic-Heun step of
Eq. S1 is differentiated along theta:

* dW/dw = W / w, dW/dalpha = -ln(1 + |i-j|) W_ij;
* the noise factor is the Cholesky factor of W(theta), so
  dL = L Phi(L^-1 dW L^-T) with Phi = lower triangle, diagonal halved (the
  standard derivative of the Cholesky factorisation); alpha = 0 and alpha = inf
  use their closed-form factors (dL = dW / (2 sqrt w) entrywise on the
  non-zero pattern);
* increments, predictor, corrector, renormalisation and the window moments are
  differentiated term by term (product rule on Eq. S1).

The objective is a linear form J = sum_k c_k mu_k of the ensemble means mu of
the window moments (S^z, A, A^2, A S^z, (S^z)^2); c for <S+S-> and for g2 follow
from the normal-ordering formulas of Sec. S1. The tangent returns dJ/dtheta,
with per-trajectory contributions for a standard error.
"""
import math

import numpy as np
import scipy.linalg

from .twa_oracle import TWAOracle, noise_factor, pump_matrix

OBJECTIVES = ("SpSm", "g2")


def pump_derivative(N, alpha, w, theta):
    """dW/dtheta for theta = 'w' or 'alpha'."""
    W = pump_matrix(N, alpha, w)
    if theta == "w":
        return W / w
    if theta == "alpha":
        d = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :]).astype(np.float64)
        return -np.log1p(d) * W
    raise ValueError(theta)


def factor_derivative(L, dW, alpha, w):
    """dL for L L^T = W along dW (Cholesky derivative; closed forms at alpha = 0, inf)."""
    N = L.shape[0]
    if w == 0.0:
        return np.zeros_like(L)
    if alpha == 0.0 or math.isinf(alpha):
        # L = sqrt(W) on its non-zero pattern (rank one column or diagonal)
        mask = L != 0.0
        out = np.zeros_like(L)
        out[mask] = dW[mask] / (2.0 * L[mask])
        return out
    X = scipy.linalg.solve_triangular(L, dW, lower=True)            # L^-1 dW
    X = scipy.linalg.solve_triangular(L, X.T, lower=True).T         # L^-1 dW L^-T
    Phi = np.tril(X)
    Phi[np.diag_indices(N)] *= 0.5
    return L @ Phi


def objective_coefficients(mu, objective):
    """c with J = sum_k c_k mu_k to first order, mu = (S^z, A, A^2, A S^z, (S^z)^2) means."""
    Sz, A, A2, ASz, Sz2 = mu
    dspsm = np.array([0.5, 1.0, 0.0, 0.0, 0.0])
    if objective == "SpSm":
        return dspsm, A + 0.5 * Sz
    if objective == "g2":
        spsm = A + 0.5 * Sz
        g2num = A2 + 2.0 * ASz - Sz / 3.0 + 0.5 * Sz2 - 4.0 / 3.0 * A
        dg2num = np.array([-1.0 / 3.0, -4.0 / 3.0, 1.0, 2.0, 0.5])
        return dg2num / spsm ** 2 - 2.0 * g2num / spsm ** 3 * dspsm, g2num / spsm ** 2
    raise ValueError(objective)


class TWATangent(TWAOracle):
    """The oracle integrator carrying a tangent (dsx, dsy, dsz) along theta."""

    def __init__(self, N, alpha, w, Gamma, dt, seed, M, theta, **kw):
        super().__init__(N, alpha, w, Gamma, dt, seed, M, **kw)
        self.theta = theta
        self.dW = pump_derivative(self.N, self.alpha, self.w, theta)
        self.dL = factor_derivative(self.L, self.dW, self.alpha, self.w)
        self.tx = np.zeros((self.M, self.N))
        self.ty = np.zeros((self.M, self.N))
        self.tz = np.zeros((self.M, self.N))
        self.dmom = np.zeros((self.M, 5))     # window sums of d phi_k

    def increment_tangent(self, s, ts, dxi, dchi, tdchi):
        """Increment of Eq. S1 and its derivative along theta (product rule)."""
        G, dt = self.Gamma, self.dt
        sx, sy, sz = s
        tx, ty, tz = ts
        dxi_x, dxi_y = dxi
        dchi_x, dchi_y = dchi
        tchi_x, tchi_y = tdchi
        Sx, Sy = sx.sum(1, keepdims=True), sy.sum(1, keepdims=True)
        tSx, tSy = tx.sum(1, keepdims=True), ty.sum(1, keepdims=True)
        Px, Py = sx @ self.W.T, sy @ self.W.T
        tPx = tx @ self.W.T + sx @ self.dW.T                     # d(W s) = W ds + dW s
        tPy = ty @ self.W.T + sy @ self.dW.T
        dx = (0.5 * G * sz * Sx - 0.5 * sz * Px) * dt + dxi_x * sz - dchi_x * sz
        dy = (0.5 * G * sz * Sy - 0.5 * sz * Py) * dt + dxi_y * sz - dchi_y * sz
        dz = (-0.5 * G * (sx * Sx + sy * Sy) + 0.5 * (sx * Px + sy * Py)) * dt \
            - (dxi_x * sx + dxi_y * sy) + (dchi_x * sx + dchi_y * sy)
        tdx = (0.5 * G * (tz * Sx + sz * tSx) - 0.5 * (tz * Px + sz * tPx)) * dt \
            + dxi_x * tz - (tchi_x * sz + dchi_x * tz)
        tdy = (0.5 * G * (tz * Sy + sz * tSy) - 0.5 * (tz * Py + sz * tPy)) * dt \
            + dxi_y * tz - (tchi_y * sz + dchi_y * tz)
        tdz = (-0.5 * G * (tx * Sx + sx * tSx + ty * Sy + sy * tSy)
               + 0.5 * (tx * Px + sx * tPx + ty * Py + sy * tPy)) * dt \
            - (dxi_x * tx + dxi_y * ty) + (tchi_x * sx + dchi_x * tx + tchi_y * sy + dchi_y * ty)
        return (dx, dy, dz), (tdx, tdy, tdz)

    def step(self):
        t = self.t
        xi_x, xi_y, eta_x, eta_y = self.noise(t)
        sg, sd = math.sqrt(self.Gamma * self.dt), math.sqrt(self.dt)
        dxi = (sg * xi_x[:, None], sg * xi_y[:, None])
        dchi = (sd * (eta_x @ self.L.T), sd * (eta_y @ self.L.T))
        tdchi = (sd * (eta_x @ self.dL.T), sd * (eta_y @ self.dL.T))
        s = (self.sx, self.sy, self.sz)
        ts = (self.tx, self.ty, self.tz)
        f, tf = self.increment_tangent(s, ts, dxi, dchi, tdchi)
        p = tuple(a + b for a, b in zip(s, f))
        tp = tuple(a + b for a, b in zip(ts, tf))
        g, tg = self.increment_tangent(p, tp, dxi, dchi, tdchi)
        u = tuple(a + 0.5 * (b + c) for a, b, c in zip(s, f, g))
        tu = tuple(a + 0.5 * (b + c) for a, b, c in zip(ts, tf, tg))
        if self.renormalize:
            n = np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
            dot = u[0] * tu[0] + u[1] * tu[1] + u[2] * tu[2]
            k = math.sqrt(3.0)
            new = tuple(k * a / n for a in u)
            tnew = tuple(k * (ta / n - a * dot / n ** 3) for a, ta in zip(u, tu))
        else:
            new, tnew = u, tu
        self.sx, self.sy, self.sz = new
        self.tx, self.ty, self.tz = tnew
        self.t = t + 1
        if self.t > self.n_window and (self.t - self.n_window) % self.sample_stride == 0:
            self.accumulate()

    def accumulate(self):
        super().accumulate()
        Sx, Sy, Sz = self.sx.sum(1), self.sy.sum(1), self.sz.sum(1)
        tSx, tSy, tSz = self.tx.sum(1), self.ty.sum(1), self.tz.sum(1)
        A = 0.25 * (Sx * Sx + Sy * Sy)
        tA = 0.5 * (Sx * tSx + Sy * tSy)
        self.dmom += np.stack([tSz, tA, 2.0 * A * tA, tA * Sz + A * tSz, 2.0 * Sz * tSz], axis=1)

    def derivative(self, objective):
        """(J, dJ/dtheta, per-trajectory dJ/dtheta samples)."""
        mu = self.window_means().mean(axis=0)
        c, J = objective_coefficients(mu, objective)
        per = (self.dmom / self.count) @ c
        return J, float(per.mean()), per


def finite_difference(N, alpha, w, Gamma, dt, seed, M, steps, theta, objective, delta, **kw):
    """Central difference of J with common random numbers (same seed, counters)."""
    vals = []
    for sgn in (+1.0, -1.0):
        a2, w2 = alpha, w
        if theta == "w":
            w2 = w * (1.0 + sgn * delta)
            h = w * delta
        else:
            a2 = alpha + sgn * delta
            h = delta
        o = TWAOracle(N, a2, w2, Gamma, dt, seed, M, **kw)
        o.run(steps)
        mu = o.window_means().mean(axis=0)
        vals.append(objective_coefficients(mu, objective)[1])
    return (vals[0] - vals[1]) / (2.0 * h)


__all__ = ["pump_derivative", "factor_derivative", "objective_coefficients", "TWATangent",
           "finite_difference", "OBJECTIVES", "noise_factor"]
