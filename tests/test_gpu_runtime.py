"""Runtime behaviour of the library on the GPU: replaying the captured step
graph gives the same bits as launching the kernels one by one, profiling
records every launch, sharded trajectory offsets reproduce the unsharded run."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(prec, steps, graph, N=200, M=70, offset=0, traj=None):
    from paper_2608_10075_b300 import twa
    old = os.environ.pop("TWA_NO_GRAPH", None)
    if not graph:
        os.environ["TWA_NO_GRAPH"] = "1"
    try:
        with twa.TWA(N, 1.0, 20.0, 1.0, 1e-3, seed=4, precision=prec, traj_offset=offset) as g:
            g.run(M, steps)
            return g.get_state()
    finally:
        os.environ.pop("TWA_NO_GRAPH", None)
        if old is not None:
            os.environ["TWA_NO_GRAPH"] = old


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_graph_replay_is_bit_exact(prec):
    a = _run(prec, 12, graph=True)
    b = _run(prec, 12, graph=False)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_trajectory_shards_reproduce_one_run(prec):
    # trajectories [40, 70) run alone with traj_offset 40 equal rows 40..69 of the full run
    full = _run(prec, 6, graph=True, M=70)
    part = _run(prec, 6, graph=True, M=30, offset=40)
    for u, v in zip(full, part):
        assert np.array_equal(u[40:], v)


def test_profile_counts_launches():
    from paper_2608_10075_b300 import twa
    with twa.TWA(300, 1.0, 20.0, 1.0, 1e-3, precision="bf16x3") as g:
        g.run(130, 1)
        g.profile(True)
        g.run(130, 4)
        p = g.profile_read()
        g.profile(False)
    for k in ("noise", "noise_factor", "predict", "correct", "close"):
        assert p[k][1] == 4 and p[k][0] > 0.0
    assert p["gemm64"][1] == 0
