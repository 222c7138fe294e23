"""FP64 CPU oracle of the two-time correlation <S+(tau) S-(0)>, its spectrum
and the linewidth (arxiv 2608.10075: Sec. S1, closing part; main text,
"Observables and method").

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product library never does.

What the paper prescribes: after the steady state is prepared, every
trajectory gets two more copies, perturbed infinitesimally along x and along
y; the three copies are integrated further with identical noise. The two-time
function splits into a symmetric part, the classical average of products of
collective spins at the two times, and a commutator part obtained from the
response functions chi_AB(tau) (Kubo formula, theta(t) <[A(t), B(0)]> =
i chi_AB(t)), measured as (copy - unperturbed) / epsilon. The spectrum is
S(omega) = 2 Re int dt e^{i omega t} <S+(t) S-(0)> and the linewidth its full
width at half maximum.

Readings (the printed formulas are garbled in their normalisation):

* The perturbation of copy beta (beta = x, y) is the classical image of the
  kick delta H = eps delta(t) S^beta with S^beta = sum_k sigma_k^beta: every
  classical spin is rotated about the beta axis by the angle 2 eps
  (exp(i eps B) sigma exp(-i eps B) = sigma + i eps [B, sigma]; for B = S^x:
  delta s^y = -2 eps s^z, delta s^z = +2 eps s^y; for B = S^y: delta s^x =
  +2 eps s^z, delta s^z = -2 eps s^x). The response is then
  chi_{S^a S^beta}(tau) = (S^a_copy(tau) - S^a(tau)) / eps. A literal shift of
  s^beta by eps would give the equal-time value <S+S-> + i N / 2, not real and
  not the normal-ordered estimator of Sec. S1 item 6.
* With S^+ = (S^x + i S^y) / 2 (sigma^+ = (sigma^x + i sigma^y) / 2),
  <S+(tau) S-(0)> = 1/4 <(S^x(tau) + i S^y(tau)) (S^x(0) - i S^y(0))>_cl
                  + i/8 (chi_xx + chi_yy + i chi_yx - i chi_xy),
  chi_ab = chi_{S^a S^b}. At tau -> 0+ this is A + <S^z>/2, the equal-time
  estimator of Sec. S1 item 6 (exactly, up to O(eps)): the normalisation is
  fixed by that limit.
* The kick happens after step `prep_steps` (time t0 = prep_steps dt); lag k
  is the state after prep_steps + k steps; C is recorded every `lag_stride`
  steps, lag 0 being the kicked state itself.
* S(omega) = 2 Re sum_k c_k e^{i omega tau_k} C(tau_k) dtau over the recorded
  lags, c_k the trapezoid weights (1/2 at both ends), i.e. the one-sided
  transform over the measured interval [0, tau_max] (C(-tau) = C(tau)* for a
  stationary process, so it is the two-sided transform).
* FWHM: the grid maximum of S, then on each side the first grid interval where
  S falls to half of it, the crossing by linear interpolation; the width is the
  distance of the two crossings (NaN if a side never falls to half).
* Standard errors: delete-one block jackknife over min(32, M) contiguous
  trajectory blocks, the whole estimator (means, spectrum, width) recomputed
  per block.
"""
import math

import numpy as np

from oracle.twa_oracle import TWAOracle

__all__ = ["kick", "two_time_samples", "correlation_from_parts", "spectrum", "fwhm", "two_time"]


def kick(sx, sy, sz, axis, eps):
    """Every spin rotated about `axis` ("x" or "y") by the angle 2 eps: the
    classical image of the kick eps delta(t) S^axis (see the module notes)."""
    c, s = math.cos(2.0 * eps), math.sin(2.0 * eps)
    if axis == "x":
        return sx.copy(), c * sy - s * sz, s * sy + c * sz
    if axis == "y":
        return c * sx + s * sz, sy.copy(), -s * sx + c * sz
    raise ValueError("axis must be 'x' or 'y'")


def _collective(o):
    return o.sx.sum(axis=1), o.sy.sum(axis=1)


def two_time_samples(N, alpha, w, Gamma, dt, seed, M, prep_steps, lag_steps, lag_stride, eps,
                     oracle_cls=TWAOracle, **kw):
    """Per-trajectory samples of the eight two-time quantities at every recorded
    lag: array (n_lags, M, 8) holding
        S^x(t) S^x(t0), S^y(t) S^y(t0), S^x(t) S^y(t0), S^y(t) S^x(t0),
        chi_xx, chi_yx, chi_xy, chi_yy
    (chi_ab = (S^a of the copy kicked by S^b - S^a) / eps), t = t0 + lag dt.
    Copy B carries the S^x kick, copy C the S^y kick; all three copies use the
    same seed, trajectory indices and step counter, hence the same noise."""
    A = oracle_cls(N, alpha, w, Gamma, dt, seed, M, **kw)
    A.run(prep_steps)
    B = oracle_cls(N, alpha, w, Gamma, dt, seed, M, W=A.W, L=A.L, **kw)
    C = oracle_cls(N, alpha, w, Gamma, dt, seed, M, W=A.W, L=A.L, **kw)
    B.sx, B.sy, B.sz = kick(A.sx, A.sy, A.sz, "x", eps)
    C.sx, C.sy, C.sz = kick(A.sx, A.sy, A.sz, "y", eps)
    B.t = C.t = A.t
    X0, Y0 = _collective(A)
    out = []

    def record():
        Xa, Ya = _collective(A)
        Xb, Yb = _collective(B)
        Xc, Yc = _collective(C)
        out.append(np.stack([Xa * X0, Ya * Y0, Xa * Y0, Ya * X0,
                             (Xb - Xa) / eps, (Yb - Ya) / eps, (Xc - Xa) / eps, (Yc - Ya) / eps], axis=1))

    record()
    for k in range(1, lag_steps + 1):
        for o in (A, B, C):
            o.run(1)
        if k % lag_stride == 0:
            record()
    return np.stack(out)


def correlation_from_parts(p):
    """<S+(tau) S-(0)> from the ensemble means p[..., 8] of the eight quantities
    (module notes): 1/4 [(xx + yy) + i (yx - xy)] + i/8 (chi_xx + chi_yy + i chi_yx - i chi_xy)."""
    p = np.asarray(p, dtype=np.float64)
    classical = 0.25 * ((p[..., 0] + p[..., 1]) + 1j * (p[..., 3] - p[..., 2]))
    response = 0.125j * (p[..., 4] + p[..., 7] + 1j * p[..., 5] - 1j * p[..., 6])
    return classical + response


def spectrum(C, dtau, omegas):
    """S(omega) = 2 Re sum_k c_k exp(i omega tau_k) C_k dtau, trapezoid weights
    c_k over the recorded lags tau_k = k dtau."""
    C = np.asarray(C, dtype=np.complex128)
    tau = np.arange(C.shape[-1]) * dtau
    c = np.ones(C.shape[-1])
    if C.shape[-1] > 1:
        c[0] = c[-1] = 0.5
    ph = np.exp(1j * np.outer(np.asarray(omegas, dtype=np.float64), tau))   # (n_omega, n_lags)
    return 2.0 * np.real(ph @ (c * C)) * dtau


def fwhm(omegas, S):
    """Full width at half maximum of S on the grid `omegas` (module notes)."""
    S = np.asarray(S, dtype=np.float64)
    om = np.asarray(omegas, dtype=np.float64)
    k = int(np.argmax(S))
    half = 0.5 * S[k]
    left = right = math.nan
    for j in range(k, 0, -1):
        if S[j - 1] <= half:
            left = om[j - 1] + (half - S[j - 1]) / (S[j] - S[j - 1]) * (om[j] - om[j - 1])
            break
    for j in range(k, len(S) - 1):
        if S[j + 1] <= half:
            right = om[j] + (S[j] - half) / (S[j] - S[j + 1]) * (om[j + 1] - om[j])
            break
    return right - left


def two_time(N, alpha, w, Gamma, dt, seed, M, prep_steps, lag_steps, lag_stride, eps, omegas,
             blocks=32, oracle_cls=TWAOracle, **kw):
    """Ensemble means of the eight quantities per lag, C(tau), S(omega), the
    linewidth and its block-jackknife standard error."""
    smp = two_time_samples(N, alpha, w, Gamma, dt, seed, M, prep_steps, lag_steps, lag_stride, eps,
                           oracle_cls=oracle_cls, **kw)
    dtau = lag_stride * dt
    parts = smp.mean(axis=1)
    C = correlation_from_parts(parts)
    S = spectrum(C, dtau, omegas)
    width = fwhm(omegas, S)
    B = min(int(blocks), M)
    se = math.nan
    if B >= 2:
        edges = [(b * M) // B for b in range(B + 1)]
        tot = smp.sum(axis=1)
        est = []
        for b in range(B):
            part_b = (tot - smp[:, edges[b]:edges[b + 1]].sum(axis=1)) / (M - (edges[b + 1] - edges[b]))
            est.append(fwhm(omegas, spectrum(correlation_from_parts(part_b), dtau, omegas)))
        est = np.asarray(est)
        se = float(math.sqrt((B - 1) / B * np.sum((est - est.mean()) ** 2)))
    return {"parts": parts, "C": C, "S": S, "fwhm": width, "fwhm_se": se, "samples": smp}
