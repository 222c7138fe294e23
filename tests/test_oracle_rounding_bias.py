"""Where the bias of the single-term precisions comes from (CPU).

The FP64 oracle is run with one operand rounded to BF16 the way a single-term
tensor-core contraction rounds it (round to nearest even after FP32), paired
with the unrounded run on the same noise. Rounding the noise factor L moves
<S^z> by far more than rounding the pump matrix W: the rows of the Cholesky
factor of a Toeplitz W converge to one sequence, so L's rounding errors repeat
on every row and change every site's pump-noise variance sum_j L_ij^2 by a
first-order amount of one sign, while W's errors enter the deterministic field
only.
"""
import math

import numpy as np

from oracle.twa_oracle import TWAOracle


def _bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _paired_sz_shift(N, alpha, w, dt, M, T, which):
    steps = int(round(T / dt))
    ref = TWAOracle(N, alpha, w, 1.0, dt, 0, M, window_start=T / 2)
    ref.run(steps)
    o = TWAOracle(N, alpha, w, 1.0, dt, 0, M, window_start=T / 2)
    if which == "L":
        o.L = _bf16(o.L)
    else:
        o.W = _bf16(o.W)
    o.run(steps)
    d = o.window_means()[:, 0] - ref.window_means()[:, 0]
    return d.mean(), d.std(ddof=1) / math.sqrt(M)


def test_rounding_the_noise_factor_dominates_the_single_term_bias():
    N, alpha, w, dt, M, T = 64, 2.0, 32.0, 2e-3, 128, 3.0
    bl, sl = _paired_sz_shift(N, alpha, w, dt, M, T, "L")
    bw, sw = _paired_sz_shift(N, alpha, w, dt, M, T, "W")
    assert abs(bl) > 10.0 * sl, (bl, sl)            # a systematic shift, not sampling noise
    assert abs(bl) > 4.0 * (abs(bw) + 2.0 * sw), (bl, bw, sw)
    # and the rounded factor changes the per-site noise variance by a one-signed amount
    from oracle.twa_oracle import noise_factor, pump_matrix
    L, W = noise_factor(N, alpha, w), pump_matrix(N, alpha, w)
    dv = (np.sum(_bf16(L) ** 2, axis=1) - np.diag(W)) / np.diag(W)
    inner = dv[N // 4: 3 * N // 4]
    assert np.all(np.sign(inner) == np.sign(inner.mean())) and abs(inner.mean()) > 1e-5
