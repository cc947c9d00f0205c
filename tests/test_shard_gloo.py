"""The sharded search's host logic on two CPU ranks (gloo, world size 2).

Each rank runs the library's shard code (paper_1511_01157_gb300.shard:
the contiguous split of the trajectory index, the gather over
torch.distributed, morse_topk_merge).  With no GPU here, the per-shard
search it calls is a CPU stand-in that returns the top-K of the shard's
range (the oracle's chi^2, written as records); on a GPU the same code calls
morse_grid_chi2_range.  The oracle's unsharded top-K is the check: every
rank's merged list must equal it, and the bench's max-over-ranks timing
helper must return the slowest rank's time on every rank.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import oracle as orc
    import synth
    A, *_ = orc.build_map(1.0, 1e-2, 2.0, 48, 600, 3.0, nthreads=1)
    g = orc.Grid(4, 6, 5, 4, 0.01, 0.5, -1.5, 1.5, 6.0, 40.0)
    t = synth.epoch_times(80, 5)
    At = orc.lightcurve_map(A, 2.0, t, 0.2, 15.0, 0.1, 0.9)
    F = 1.1 * At + 0.2 + 0.003 * np.sin(7 * t)
    w = np.full(len(t), 1e4)
    return orc, A, g, t, F, w


def _rank(rank, world, port, k, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    import bench
    import paper_1511_01157_gb300 as m
    w_, r_, _ = bench.dist_setup()
    assert (w_, r_) == (world, rank)
    orc, A, g, t, F, w = _problem()
    from paper_1511_01157_gb300 import shard

    def search_range(first, count):  # CPU stand-in for the GPU shard
        chi2, fs, fb, fl = orc.grid_chi2(g, t, F, w, A=A, L=2.0,
                                         first=first, count=count)
        idx, val = orc.topk(chi2, k, first=first)
        mine = shard.empty_fits(k)
        mine["chi2"][:len(idx)] = val
        mine["idx"][:len(idx)] = idx
        return mine

    merged = shard.sharded_topk(search_range, g.size, k, rank, world,
                                shard.torch_gather())
    # slowest rank's time everywhere
    tmax = bench.max_over_ranks(1.0 + rank, world)
    bench.barrier(world)
    dist.destroy_process_group()
    out_q.put((rank, merged["idx"].tolist(), merged["chi2"].tolist(), tmax))


@pytest.mark.parametrize("k", [5, 200])
def test_two_rank_shards_merge_to_unsharded_topk(k):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, k, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    orc, A, g, t, F, w = _problem()
    chi2, *_ = orc.grid_chi2(g, t, F, w, A=A, L=2.0)
    idx, val = orc.topk(chi2, min(k, g.size))
    for rank, midx, mchi2, tmax in res:
        assert tmax == 2.0
        assert midx[:len(idx)] == idx.tolist()
        assert mchi2[:len(idx)] == val.tolist()
        assert all(i == -1 for i in midx[len(idx):])
