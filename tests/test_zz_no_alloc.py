"""The allocation-free ensemble reduction (twa_reduce_moments_noalloc).

Some callers cannot allocate device memory: a host program whose own memory
manager already owns the GPU, or a loop whose policy forbids allocation after
start-up. For them the library keeps the reduction's scratch in a fixed device
array. These tests check that entry point against the allocating one, through
the C ABI, on two calls in a row (the second smaller, so stale data left in the
shared array by the first call would show). This file is collected last.
"""
import numpy as np
import pytest

from oracle.twa_oracle import observables_from_moments

KEYS = ("Sz", "Sz_se", "sigma_z", "SpSm", "SpSm_se", "G2num", "G2num_se", "g2", "g2_se")


def _moments(M, N, seed):
    """Window means with the structure of real ones: S^z, A = |S_perp|^2/4 >= 0 and
    its powers, built from per-trajectory collective spins."""
    rng = np.random.default_rng(seed)
    Sz = rng.normal(0.3 * N, 0.2 * N, size=M)
    A = rng.gamma(3.0, N / 3.0, size=M)
    return np.column_stack([Sz, A, A * A * (1 + 0.1 * rng.random(M)), A * Sz, Sz * Sz])


@pytest.mark.gpu
def test_noalloc_matches_allocating_reduction_twice():
    from paper_2608_10075_b300 import twa
    N = 300
    for call, M in enumerate((5000, 1234)):
        means = _moments(M, N, seed=call)
        ref = twa.reduce_moments(means, N)
        got = twa.reduce_moments_noalloc(means, N)
        for k in KEYS:
            assert abs(got[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (call, k, got[k], ref[k])
        assert got["M"] == M
        # and both agree with the oracle's reduction of the same samples
        orc = observables_from_moments(means, N)
        for k in ("Sz", "SpSm", "G2num", "g2", "g2_se"):
            assert abs(got[k] - orc[k]) <= 1e-9 * max(1.0, abs(orc[k])), (k, got[k], orc[k])


def test_noalloc_rejects_more_than_its_scratch_holds():
    from paper_2608_10075_b300 import twa
    means = np.zeros((twa.NOALLOC_MAX_M + 1, 5))
    with pytest.raises(twa.TWAError) as e:
        twa.reduce_moments_noalloc(means, 10)
    assert e.value.code == -1 and "TWA_NOALLOC_MAX_M" in str(e.value)
    with pytest.raises(twa.TWAError):
        twa.reduce_moments_noalloc(np.zeros((0, 5)), 10)
