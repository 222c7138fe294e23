"""The allocation-free ensemble reduction (twa_reduce_moments_noalloc).

Some callers cannot allocate device memory: a host program whose own memory
manager already owns the GPU, or a loop whose policy forbids allocation after
start-up. For them the library keeps the reduction's scratch in a fixed device
array. These tests check that entry point against the allocating one, through
the C ABI, on two calls in a row (the second smaller, so stale data left in the
shared array by the first call would show). This file is collected last.
"""
import json
import os
import subprocess
import sys

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


# Runs in a child process: reductions in the primary context, then in a context
# the child creates itself with the driver API (as a host application with its
# own CUDA set-up would), then in the primary context again. The scratch array
# has a different device address in each context, which the entry point must
# look up in the context that is current at the call.
_CONTEXT_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from cuda.bindings import driver as cu
from paper_2608_10075_b300 import twa
from tests.test_zz_no_alloc import _moments

def ok(r):
    err = r[0] if isinstance(r, tuple) else r
    assert int(err) == 0, err
    return r[1] if isinstance(r, tuple) and len(r) > 1 else None

N = 64
out = []
means = _moments(3000, N, seed=7)
out.append(("primary", twa.reduce_moments(means, N), twa.reduce_moments_noalloc(means, N)))
ok(cu.cuInit(0))
dev = ok(cu.cuDeviceGet(0))
ctx = ok(cu.cuCtxCreate(None, 0, dev))
means2 = _moments(777, N, seed=8)
own = twa.reduce_moments_noalloc(means2, N)
ok(cu.cuCtxPopCurrent())
ok(cu.cuCtxDestroy(ctx))
out.append(("own context", twa.reduce_moments(means2, N), own))
means3 = _moments(1500, N, seed=9)
out.append(("primary again", twa.reduce_moments(means3, N), twa.reduce_moments_noalloc(means3, N)))
print(json.dumps(out))
"""


@pytest.mark.gpu
def test_noalloc_in_a_caller_created_context():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CONTEXT_CHILD, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    for where, ref, got in json.loads(r.stdout.strip().splitlines()[-1]):
        for k in KEYS:
            assert abs(got[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (where, k, got[k], ref[k])


def test_noalloc_rejects_more_than_its_scratch_holds():
    from paper_2608_10075_b300 import twa
    means = np.zeros((twa.NOALLOC_MAX_M + 1, 5))
    with pytest.raises(twa.TWAError) as e:
        twa.reduce_moments_noalloc(means, 10)
    assert e.value.code == -1 and "TWA_NOALLOC_MAX_M" in str(e.value)
    with pytest.raises(twa.TWAError):
        twa.reduce_moments_noalloc(np.zeros((0, 5)), 10)
