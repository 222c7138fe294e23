"""Sharded ensembles on several ranks, on the CPU with gloo (world size 2 and 3).

Each rank integrates its share of trajectories with the oracle (standing in for
one GPU's engine: the sharding logic is the same), offset in the Philox counter
as the library's traj_offset does; the per-trajectory window means are gathered
with paper_2608_10075_b300.ensemble and must equal, row for row, a single run
over all trajectories.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2608_10075_b300.ensemble import gather_means, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, M_total, out_dir):
    import torch.distributed as dist
    from oracle.twa_oracle import TWAOracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, cnt = shard(M_total, world, rank)
    o = TWAOracle(9, 1.0, 4.0, 1.0, 2e-3, 17, cnt, m0=off, window_start=0.02)
    o.run(25)
    full = gather_means(o.window_means())
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_partition():
    for M_total, world in ((10, 3), (7, 7), (5, 2), (1024, 8)):
        spans = [shard(M_total, world, r) for r in range(world)]
        assert spans[0][0] == 0
        for (o1, c1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + c1 == o2
        assert sum(c for _, c in spans) == M_total


@pytest.mark.parametrize("world", [2, 3])
def test_gathered_shards_equal_one_run(world, tmp_path):
    from oracle.twa_oracle import TWAOracle
    M_total = 11
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, M_total, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(os.path.join(tmp_path, "gathered.npy"))
    ref = TWAOracle(9, 1.0, 4.0, 1.0, 2e-3, 17, M_total, window_start=0.02)
    ref.run(25)
    assert got.shape == (M_total, 5)
    # BLAS may sum a row in another order for another batch size: rounding only
    assert np.allclose(got, ref.window_means(), rtol=1e-12, atol=0)
