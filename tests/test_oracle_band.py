"""Why the two-product band of BF16L2 and BF16B removes the one-term bias (CPU).

The tensor-core images hold W / w and L / sqrt(w) in BF16. With one product per
entry, each entry carries its BF16 rounding error. W is Toeplitz, so the error
of each diagonal offset d = |i - j| repeats on every row, and the rows of the
Cholesky factor L converge to one sequence: the errors add up to a row sum of
one sign on every row. The steady state feels that row sum through the pump
field (W) and through each site's pump-noise variance sum_j L_ij^2 (L). Taking
hi + lo on the band j in [u - 64, u + 320) of the rows i in [u, u + 256) (u a
multiple of 256) keeps the largest entries, which dominate those sums, to ~2^-16.

These tests pin that mechanism on the oracle's matrices with the BF16 rounding
emulated: the band's geometry, the one-signed one-term sums, and what is left
off the band (for W at alpha = 1 and 2, and for L at every alpha; at alpha = 0.5
the slowly decaying tail of W keeps its row sums, where the measured ensembles
show no bias).
"""
import numpy as np
import pytest

from oracle.twa_oracle import noise_factor
from tests.mixed_bounds import bf16


def band_mask(N):
    """True where entry (i, j) takes two products: j in [u - 64, u + 320), u = 256 floor(i / 256)."""
    i = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    u = (i // 256) * 256
    return (j >= u - 64) & (j < u + 320)


def test_band_holds_every_entry_within_64_of_the_diagonal():
    N = 1000
    band = band_mask(N)
    d = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :])
    assert np.all(band[d <= 64])
    # and at most 384 columns per row: 3.8 % of W's entries at N = 10^4
    assert band.sum(axis=1).max() == 384


def _w_row_error_sums(N, alpha):
    """Per row i of W / w = 1 / (1 + |i - j|)^alpha: the sum of the one-term BF16
    rounding errors over all j, and over the j off the band (Toeplitz: from the
    error of each offset and its prefix sums)."""
    d = np.arange(N, dtype=np.float64)
    v = 1.0 / (1.0 + d) ** alpha
    e = bf16(v) - v
    cs = np.concatenate([[0.0], np.cumsum(e)])      # cs[k] = e[0] + ... + e[k - 1]
    i = np.arange(N)
    full = cs[i + 1] + cs[N - i] - e[0]              # offsets 0..i to the left, 0..N-1-i to the right
    u = (i // 256) * 256
    lo, hi = np.maximum(u - 64, 0), np.minimum(u + 320, N)
    inband = cs[i - lo + 1] + cs[hi - i] - e[0]
    return full, full - inband


@pytest.mark.parametrize("alpha,shrink", [(1.0, 20.0), (2.0, 300.0)])
def test_one_term_w_row_sums_are_one_signed_and_the_band_removes_them(alpha, shrink):
    full, off = _w_row_error_sums(10000, alpha)
    # one product everywhere: the same sign on every row, none near zero
    assert np.all(full > 0.0) or np.all(full < 0.0)
    assert np.min(np.abs(full)) > 0.3 * np.max(np.abs(full))
    # off the band what is left is a small fraction of it
    assert np.max(np.abs(off)) < np.max(np.abs(full)) / shrink


def test_w_tail_keeps_its_row_sums_at_alpha_half():
    # at alpha = 0.5 W decays slowly and the entries beyond the band carry row
    # sums as large as the one-term ones: the band does not shrink them
    full, off = _w_row_error_sums(10000, 0.5)
    assert np.max(np.abs(off)) > 0.5 * np.max(np.abs(full))


@pytest.mark.parametrize("alpha,shrink", [(0.5, 30.0), (1.0, 1000.0), (2.0, 1e5)])
def test_one_term_l_noise_variance_error_is_one_signed_and_the_band_removes_it(alpha, shrink):
    N = 1024
    L = noise_factor(N, alpha, 1.0)                  # the image L / sqrt(w)
    d2 = bf16(L) ** 2 - L ** 2                       # one product: per-entry error of L_ij^2
    var = (L ** 2).sum(axis=1)
    full = d2.sum(axis=1) / var                      # relative error of each site's noise variance
    off = np.where(band_mask(N), 0.0, d2).sum(axis=1) / var
    rows = slice(256, N)                             # rows past the first unit, whose L has converged
    assert np.all(full[rows] < 0.0)                  # less pump noise on every site
    assert np.max(np.abs(off[rows])) < np.max(np.abs(full[rows])) / shrink
