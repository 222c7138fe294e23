"""Sharded ensemble through the library itself: two gloo ranks (child processes
on the one GPU, each with its own context; no kernel of one rank waits on the
other, the only exchange is the host-side gather at the end) run their shares
of the trajectories with traj_offset, gather the per-trajectory window means
with paper_2608_10075_b300.ensemble and reduce them with twa_reduce_moments.
Trajectories depend only on their Philox indices, so the gathered means equal
an unsharded run row for row and the observables are identical."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

CASE = dict(N=300, alpha=1.0, w=40.0, Gamma=1.0, dt=5e-4, precision="bf16x2", window_start=0.01)
STEPS, M_TOTAL = 40, 300


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2608_10075_b300 import twa
    from paper_2608_10075_b300.ensemble import gather_means, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, cnt = shard(M_TOTAL, world, rank)
    c = CASE
    with twa.TWA(c["N"], c["alpha"], c["w"], c["Gamma"], c["dt"], seed=3, precision=c["precision"],
                 window_start=c["window_start"], traj_offset=off) as g:
        g.run(cnt, STEPS)
        local = g.moments()
    full = gather_means(local)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), full)
        obs = twa.reduce_moments(full, c["N"])
        np.save(os.path.join(out_dir, "obs.npy"), np.array([obs[k] for k in ("Sz", "SpSm", "G2num", "g2", "g2_se")]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reproduce_one_run(tmp_path):
    from paper_2608_10075_b300 import twa
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(os.path.join(tmp_path, "gathered.npy"))
    c = CASE
    with twa.TWA(c["N"], c["alpha"], c["w"], c["Gamma"], c["dt"], seed=3, precision=c["precision"],
                 window_start=c["window_start"]) as g:
        g.run(M_TOTAL, STEPS)
        ref = g.moments()
        ob = g.observables()
    assert got.shape == (M_TOTAL, 5)
    assert np.array_equal(got, ref)
    obs = np.load(os.path.join(tmp_path, "obs.npy"))
    for v, k in zip(obs, ("Sz", "SpSm", "G2num", "g2", "g2_se")):
        assert abs(v - ob[k]) <= 1e-12 * max(1.0, abs(ob[k])), (k, v, ob[k])
