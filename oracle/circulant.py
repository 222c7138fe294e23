"""FP64 CPU oracle for the circulant-embedding draw of the correlated pump noise.

TEST INFRASTRUCTURE, like ``twa_oracle``: only ``tests/``, ``__graft_entry__``
and the CPU legs of ``bench.py`` may import it; the product library never does.

What it follows (arxiv 2608.10075): the pump noise of Eq. (S1) has correlator
<chi_i^a chi_j^b> = w_ij delta_ab with w_ij of Eq. (2), which depends only on
|i - j|. Any Gaussian vector with covariance W gives the same law; the Cholesky
draw chi = L eta (``twa_oracle``) is one, this module is another:

* Embedding (Dietrich & Newsam, SIAM J. Sci. Comput. 18 (1997); Wood & Chan,
  J. Comput. Graph. Stat. 3 (1994)): on a circle of even length P >= 2N - 2,
  the sequence c_d = w / (1 + min(d, P - d))^alpha, d = 0 .. P-1, is the first
  row of a symmetric circulant C whose leading N x N block is W (every |i - j|
  < N is at most P / 2). For alpha >= 0 the sequence is non-negative,
  non-increasing and convex on 0 .. P/2, which makes C positive semi-definite:
  its eigenvalues lam_k = sum_d c_d cos(2 pi k d / P) are >= 0.
* Draw: with Z_k = a_k + i b_k, a_k, b_k independent standard normals,
  Y_j = sum_k sqrt(lam_k / P) Z_k exp(+2 pi i j k / P). Re Y and Im Y are two
  independent Gaussian vectors, each with covariance C, so chi^x_j = Re Y_j and
  chi^y_j = Im Y_j (j < N) are the two pump-noise components with covariance W.
* Random stream: (a_k, b_k) are the Box-Muller pair of the Philox4x32-10 call
  at counter (trajectory m, step t, frequency k, stream 2); the collective noise
  xi keeps its counter (m, t, N, stream 0).
* Length: P is the smallest even 2^a 3^b 5^c with P >= max(2, 2N - 2), or a
  given even P >= 2N - 2 (any such circle gives a valid embedding; the library
  takes a multiple of 4 C when C CTAs share one transform and reports P).

A library FFT (numpy.fft) serves as the transform; the tests pin it against the
sums above written out term by term.
"""
import math

import numpy as np

from oracle.twa_oracle import TWAOracle, philox_normals

__all__ = ["embedding_length", "embedded_sequence", "embedding_spectrum", "circulant_chi",
           "TWAOracleCirculant"]

STREAM_CIRCULANT = 2


def _smooth(v):
    for f in (2, 3, 5):
        while v % f == 0:
            v //= f
    return v == 1


def embedding_length(N):
    """Smallest even 5-smooth P with P >= max(2, 2N - 2)."""
    P = max(2, 2 * int(N) - 2)
    while P % 2 or not _smooth(P):
        P += 1
    return P


def embedded_sequence(N, alpha, w, P):
    """First row of the circulant embedding of Eq. (2): c_d = w / (1 + min(d, P-d))^alpha."""
    d = np.arange(P)
    dist = np.minimum(d, P - d).astype(np.float64)
    if math.isinf(alpha):
        return np.where(dist == 0, float(w), 0.0)
    return float(w) / np.power(dist + 1.0, alpha)


def embedding_spectrum(c):
    """lam_k = sum_d c_d exp(-2 pi i k d / P); real because c is symmetric."""
    return np.fft.fft(c).real


def circulant_chi(seed, m, t, N, lam):
    """(chi^x, chi^y), each of shape (len(m), N), for trajectories m at step t.

    m: 1-D array of global trajectory indices; lam: the embedding spectrum.
    """
    P = lam.shape[0]
    mm = np.asarray(m, dtype=np.uint64)[:, None]
    kk = np.arange(P, dtype=np.uint64)[None, :]
    a, b = philox_normals(seed, mm, np.uint64(t), kk, STREAM_CIRCULANT)
    scale = np.sqrt(np.maximum(lam, 0.0) / P)
    # Y_j = sum_k scale_k Z_k exp(+2 pi i j k / P) = P * ifft(scale * Z)
    Y = P * np.fft.ifft(scale[None, :] * (a + 1j * b), axis=1)
    return Y.real[:, :N].copy(), Y.imag[:, :N].copy()


class TWAOracleCirculant(TWAOracle):
    """``TWAOracle`` with the pump noise drawn through the circulant embedding
    instead of the Cholesky factor (same law, different per-trajectory values)."""

    def __init__(self, N, alpha, w, Gamma, dt, seed, M, P=None, **kw):
        # this draw needs no factor of W: skip the base class's Cholesky
        kw.setdefault("L", np.zeros((0, 0)))
        super().__init__(N, alpha, w, Gamma, dt, seed, M, **kw)
        self.P = embedding_length(self.N) if P is None else int(P)
        if self.P % 2 or self.P < max(2, 2 * self.N - 2):
            raise ValueError("the circle length must be even and >= 2N - 2")
        self.lam = embedding_spectrum(embedded_sequence(self.N, self.alpha, self.w, self.P))

    def noise_increments(self, t):
        xi_x, xi_y, _, _ = self.noise(t)
        sg = math.sqrt(self.Gamma * self.dt)
        sd = math.sqrt(self.dt)
        chi_x, chi_y = circulant_chi(self.seed, self.m0 + np.arange(self.M), t, self.N, self.lam)
        return sg * xi_x[:, None], sg * xi_y[:, None], sd * chi_x, sd * chi_y
