"""Pins of the circulant-embedding noise oracle (CPU).

The draw must give the pump noise of Eq. (S1) a covariance equal to w_ij of
Eq. (2). These tests check that law without the oracle's FFT: the linear map
from the 2P Philox normals to chi is written out here term by term from its
definition, its Gram matrix must be W exactly (to rounding), and the oracle's
FFT-based draw must equal that map applied to the same normals.
"""
import math

import numpy as np
import pytest

from oracle.circulant import (TWAOracleCirculant, circulant_chi, embedded_sequence, embedding_length,
                              embedding_spectrum)
from oracle.twa_oracle import TWAOracle, philox_normals, pump_matrix


def _is_smooth(v):
    for f in (2, 3, 5):
        while v % f == 0:
            v //= f
    return v == 1


@pytest.mark.parametrize("N", [1, 2, 3, 5, 16, 37, 38, 300, 1024, 5001, 10000, 14001])
def test_embedding_length_is_the_smallest_even_smooth_bound(N):
    P = embedding_length(N)
    lo = max(2, 2 * N - 2)
    assert P >= lo and P % 2 == 0 and _is_smooth(P)
    assert not any(q % 2 == 0 and _is_smooth(q) for q in range(lo, P))


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0, 2.0, math.inf])
@pytest.mark.parametrize("N", [1, 4, 9, 38])
def test_leading_block_of_the_circulant_is_W(N, alpha):
    P = embedding_length(N)
    c = embedded_sequence(N, alpha, 3.0, P)
    idx = np.arange(N)
    C = c[(idx[:, None] - idx[None, :]) % P]
    assert np.array_equal(C, pump_matrix(N, alpha, 3.0))
    # symmetric circle: c_d = c_{P - d}
    assert np.array_equal(c[1:], c[1:][::-1])


@pytest.mark.parametrize("N,alpha", [(4, 1.0), (7, 0.5), (12, 2.0), (1, 1.0), (9, 0.0), (6, math.inf)])
def test_spectrum_is_the_cosine_sum(N, alpha):
    P = embedding_length(N)
    c = embedded_sequence(N, alpha, 2.5, P)
    lam = embedding_spectrum(c)
    ref = [sum(c[d] * math.cos(2.0 * math.pi * k * d / P) for d in range(P)) for k in range(P)]
    assert np.allclose(lam, ref, rtol=0, atol=1e-12 * max(1.0, max(abs(x) for x in ref)))


@pytest.mark.parametrize("alpha", [0.0, 0.1, 0.25, 0.5, 1.0, 2.0, 3.0, math.inf])
@pytest.mark.parametrize("N", [1, 2, 5, 16, 37, 300, 1024, 10000])
def test_spectrum_is_nonnegative(N, alpha):
    # Dietrich-Newsam: non-negative, non-increasing, convex on 0..P/2 => PSD
    P = embedding_length(N)
    lam = embedding_spectrum(embedded_sequence(N, alpha, 1.0, P))
    assert lam.min() >= -1e-12 * lam.max()


def _explicit_map(N, alpha, w, P=None):
    """Real N x 2P matrices Ax, Ay with chi^x = Ax [a; b], chi^y = Ay [a; b],
    from Y_j = sum_k sqrt(lam_k / P) (a_k + i b_k) (cos + i sin)(2 pi j k / P)."""
    P = embedding_length(N) if P is None else P
    c = embedded_sequence(N, alpha, w, P)
    lam = [sum(c[d] * math.cos(2.0 * math.pi * k * d / P) for d in range(P)) for k in range(P)]
    Ax = np.zeros((N, 2 * P))
    Ay = np.zeros((N, 2 * P))
    for j in range(N):
        for k in range(P):
            s = math.sqrt(max(lam[k], 0.0) / P)
            th = 2.0 * math.pi * j * k / P
            Ax[j, k], Ax[j, P + k] = s * math.cos(th), -s * math.sin(th)
            Ay[j, k], Ay[j, P + k] = s * math.sin(th), s * math.cos(th)
    return Ax, Ay


@pytest.mark.parametrize("N,alpha,w", [(1, 1.0, 2.0), (5, 1.0, 3.0), (6, 0.5, 1.0), (7, 2.0, 4.0), (8, 0.0, 2.0),
                                       (9, math.inf, 1.5), (13, 0.25, 1.0)])
def test_draw_has_covariance_W(N, alpha, w):
    Ax, Ay = _explicit_map(N, alpha, w)
    W = pump_matrix(N, alpha, w)
    tol = 1e-12 * w * Ax.shape[1]
    assert np.allclose(Ax @ Ax.T, W, rtol=0, atol=tol)
    assert np.allclose(Ay @ Ay.T, W, rtol=0, atol=tol)
    assert np.allclose(Ax @ Ay.T, 0.0, rtol=0, atol=tol)   # independent components


@pytest.mark.parametrize("N,alpha,w,P", [(5, 1.0, 3.0, 16), (7, 0.5, 1.0, 32), (9, 2.0, 4.0, 24), (6, 0.0, 2.0, 40),
                                         (4, math.inf, 1.0, 8)])
def test_any_longer_even_circle_has_covariance_W(N, alpha, w, P):
    # the cluster form of the library takes P a multiple of 4 C, not always the
    # smallest even smooth bound: the embedding on any even P >= 2N - 2 is exact
    assert P % 2 == 0 and P > embedding_length(N)
    Ax, Ay = _explicit_map(N, alpha, w, P)
    W = pump_matrix(N, alpha, w)
    tol = 1e-12 * w * Ax.shape[1]
    assert np.allclose(Ax @ Ax.T, W, rtol=0, atol=tol)
    assert np.allclose(Ay @ Ay.T, W, rtol=0, atol=tol)
    assert np.allclose(Ax @ Ay.T, 0.0, rtol=0, atol=tol)
    o = TWAOracleCirculant(N, alpha, w, 1.0, 1e-3, 3, 2, P=P)
    assert o.P == P and o.L.size == 0
    cx, cy = circulant_chi(3, np.array([0, 1]), 4, N, o.lam)
    a, b = philox_normals(3, np.uint64(1), np.uint64(4), np.arange(P, dtype=np.uint64), 2)
    v = np.concatenate([a, b])
    extra = 1e-6 if alpha == 0.0 else 0.0
    assert np.allclose(cx[1], Ax @ v, rtol=0, atol=1e-12 * (1 + np.abs(Ax @ v).max()) + extra)
    assert np.allclose(cy[1], Ay @ v, rtol=0, atol=1e-12 * (1 + np.abs(Ay @ v).max()) + extra)
    with pytest.raises(ValueError):
        TWAOracleCirculant(N, alpha, w, 1.0, 1e-3, 3, 2, P=2 * N - 4)


@pytest.mark.parametrize("N,alpha,w", [(5, 1.0, 3.0), (8, 0.0, 2.0), (11, 1.7, 0.5), (2, math.inf, 1.0)])
def test_oracle_draw_is_the_explicit_map_on_the_philox_normals(N, alpha, w):
    Ax, Ay = _explicit_map(N, alpha, w)
    P = embedding_length(N)
    lam = embedding_spectrum(embedded_sequence(N, alpha, w, P))
    seed, t, ms = 77, 5, np.array([0, 3, 1000])
    cx, cy = circulant_chi(seed, ms, t, N, lam)
    # alpha = 0: all but one eigenvalue vanish, and sqrt turns their rounding
    # (~1e-16 w P, computed differently here and in the FFT) into ~1e-8
    extra = 1e-6 if alpha == 0.0 else 0.0
    for r, m in enumerate(ms):
        a, b = philox_normals(seed, np.uint64(m), np.uint64(t), np.arange(P, dtype=np.uint64), 2)
        v = np.concatenate([a, b])
        assert np.allclose(cx[r], Ax @ v, rtol=0, atol=1e-12 * (1 + np.abs(Ax @ v).max()) + extra)
        assert np.allclose(cy[r], Ay @ v, rtol=0, atol=1e-12 * (1 + np.abs(Ay @ v).max()) + extra)


def test_collective_pump_noise_is_one_number_per_component():
    # alpha = 0: W = w 1 1^T has rank one, so every site gets the same chi
    N, w = 10, 2.0
    P = embedding_length(N)
    lam = embedding_spectrum(embedded_sequence(N, 0.0, w, P))
    cx, cy = circulant_chi(3, np.arange(4), 7, N, lam)
    assert np.allclose(cx, cx[:, :1], atol=1e-12) and np.allclose(cy, cy[:, :1], atol=1e-12)


def test_sample_covariance():
    N, alpha, w, M = 6, 1.0, 2.0, 40000
    P = embedding_length(N)
    lam = embedding_spectrum(embedded_sequence(N, alpha, w, P))
    cx, cy = circulant_chi(1, np.arange(M), 0, N, lam)
    W = pump_matrix(N, alpha, w)
    for c in (cx, cy):
        S = c.T @ c / M
        # entrywise SE of a sample covariance: sqrt((W_ii W_jj + W_ij^2) / M)
        se = np.sqrt((np.outer(np.diag(W), np.diag(W)) + W * W) / M)
        assert np.all(np.abs(S - W) <= 5.0 * se)
    assert np.all(np.abs(cx.T @ cy / M) <= 5.0 * np.sqrt(np.outer(np.diag(W), np.diag(W)) / M))


def test_circulant_oracle_keeps_the_collective_noise_and_the_law():
    # same xi and initial state as the Cholesky oracle; ensemble observables of
    # the two draws agree within sampling error
    N, alpha, w, G, dt, M, steps, t0 = 6, 1.0, 4.0, 1.0, 2e-3, 3000, 400, 0.4
    a = TWAOracle(N, alpha, w, G, dt, 11, M, window_start=t0)
    b = TWAOracleCirculant(N, alpha, w, G, dt, 11, M, window_start=t0)
    assert np.array_equal(a.sx, b.sx) and np.array_equal(a.sy, b.sy)
    xa = a.noise_increments(3)
    xb = b.noise_increments(3)
    assert np.array_equal(xa[0], xb[0]) and np.array_equal(xa[1], xb[1])
    assert not np.allclose(xa[2], xb[2])
    a.run(steps)
    b.run(steps)
    oa, ob = a.observables(), b.observables()
    for k in ("Sz", "SpSm", "G2num"):
        assert abs(oa[k] - ob[k]) <= 3.0 * math.hypot(oa[k + "_se"], ob[k + "_se"]), (k, oa[k], ob[k])
