"""Failure paths of the C ABI, made without any GPU fault.

* Allocation failure: a caller allocator (twa_opts.alloc) that refuses its k-th
  request, for every k a full session makes. Each must end in TWA_ENOMEM with
  every block already handed out returned (after the context is destroyed), and
  the process must still run a clean session afterwards.
* Timeout: twa_wait_probe runs the bounded mbarrier wait of the tensor-core
  kernels on a barrier that nothing completes; the next synchronising call must
  report TWA_ETIMEOUT, and a new context must still work.
* Non-positive pivots: at alpha = 1e-15 the FP64 pump matrix is numerically
  rank one with rounding noise of both signs (its smallest eigenvalue is
  negative, see the CPU test of the oracle), so the Cholesky factor meets
  non-positive pivots: TWA_ENOTPSD without clip_negative; with it, the zeroed
  columns are counted and ||W - L L^T|| / ||W|| is reported.
"""
import math

import numpy as np
import pytest

from oracle.twa_oracle import pump_matrix

pytestmark = pytest.mark.gpu


class _CountingAllocator:
    """Device memory from torch's caching allocator; refuses request `fail_at`."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.calls = 0
        self.fail_at = None

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return 0
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream))
        self.live[p] = nbytes
        return p

    def free(self, ptr, stream):
        assert ptr in self.live, "free of a pointer the allocator never handed out"
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)


def _session(twa, A, prec):
    # set-up, a run long enough to replay captured steps, observables, state to host
    with twa.TWA(37, 1.0, 3.0, 1.0, 1e-3, seed=1, precision=prec, window_start=0.002,
                 allocator=(A.alloc, A.free)) as g:
        g.run(20, 6)
        g.observables()
        g.get_state()
        g.moments()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_allocation_failure_at_every_request(prec):
    from paper_2608_10075_b300 import twa
    A = _CountingAllocator()
    _session(twa, A, prec)
    total = A.calls
    assert total > 5 and not A.live
    for k in range(1, total + 1):
        A.calls, A.fail_at = 0, k
        with pytest.raises(twa.TWAError) as e:
            _session(twa, A, prec)
        assert e.value.name == "TWA_ENOMEM", (k, str(e.value))
        assert not A.live, (k, len(A.live))
    A.calls, A.fail_at = 0, None
    _session(twa, A, prec)
    assert A.calls == total and not A.live


def test_bounded_wait_reports_timeout():
    from paper_2608_10075_b300 import twa
    with twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="bf16x3") as g:
        g.run(16, 2)
        g.sync()
        g.wait_probe(20000)   # 20 ms
        with pytest.raises(twa.TWAError) as e:
            g.sync()
        assert e.value.name == "TWA_ETIMEOUT"
        with pytest.raises(twa.TWAError) as e:
            g.observables()
        assert e.value.name == "TWA_ETIMEOUT"
    with pytest.raises(twa.TWAError) as e:
        with twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="bf16x3") as g:
            g.wait_probe(0)
    assert e.value.name == "TWA_EINVAL"
    # the device and the library stay usable
    with twa.TWA(64, 1.0, 8.0, 1.0, 1e-3, precision="bf16x3", window_start=0.001) as g:
        g.run(16, 4)
        assert math.isfinite(g.observables()["Sz"])


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_clip_negative_pivots(prec):
    from paper_2608_10075_b300 import twa
    N, alpha, w = 200, 1e-15, 5.0
    with pytest.raises(twa.TWAError) as e:
        twa.TWA(N, alpha, w, 1.0, 1e-3, precision=prec)
    assert e.value.name == "TWA_ENOTPSD"
    with twa.TWA(N, alpha, w, 1.0, 1e-3, precision=prec, clip_negative=True, window_start=0.002) as g:
        g.run(32, 5)
        ob = g.observables()
    assert ob["clipped"] >= 1 and ob["nonfinite"] == 0
    # the dropped pivots are rounding noise of a rank-one matrix: L L^T stays W
    # to the precision W itself carries
    assert 0.0 < ob["factor_residual"] < 1e-12, ob["factor_residual"]
    W = pump_matrix(N, alpha, w)
    assert np.linalg.eigvalsh(W)[0] < 0.0
