"""Multi-process source sharding on CPU (gloo, world sizes 2 and 8).

Each rank fabricates the per-source loop values of its own sources (a
deterministic function of the global source index, standing in for the GPU
solves); the gathered sets must equal those of one process that ran all
sources, in source order, and the global TSM estimate computed from them (here
with the oracle's combination standing in for tsm_combine) must equal the
single-process one bit for bit.  With 8 ranks every rank first runs the
library build step (as bench.py's ranks do): it serialises on the build lock
and leaves one library.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1401_6749_gb300.distributed import gather_tsm_sets, rank_sources

N_HP, N_LP, LEN = 3, 7, 10


def _loops_of_source(r, hp):
    """Stand-in per-source loop values (complex, as re/im doubles)."""
    rng = np.random.default_rng(1000 + 2 * r + (1 if hp else 0))
    return rng.standard_normal(2 * LEN)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path, do_build=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    if do_build:
        from paper_1401_6749_gb300 import build
        build.build()
        assert build.up_to_date()
    first, n = rank_sources(rank, N_HP, N_LP)
    hp = torch.tensor(np.stack([_loops_of_source(first + j, True) for j in range(N_HP)]))
    lp = torch.tensor(np.stack([_loops_of_source(first + j, False) for j in range(n)]))
    hp_all, lp_on_hp, lp_only = gather_tsm_sets(dist, hp, lp, N_HP)
    if rank == 0:
        np.savez(out_path, hp=hp_all.numpy(), lphp=lp_on_hp.numpy(), lp=lp_only.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_rank_sources_partition():
    ranges = [rank_sources(g, N_HP, N_LP) for g in range(4)]
    idx = [i for first, n in ranges for i in range(first, first + n)]
    assert idx == list(range(4 * (N_HP + N_LP)))


@pytest.mark.parametrize("world", [2, 8])
def test_rank_gather_matches_single_process(tmp_path, world):
    out = str(tmp_path / "gathered.npz")
    mp.spawn(_worker, args=(world, _free_port(), out, world == 8), nprocs=world, join=True)
    got = np.load(out)
    # single process: sources 0 .. world (N_HP + N_LP) - 1, HP = first N_HP of each rank
    hp, lphp, lp = [], [], []
    for g in range(world):
        first, n = rank_sources(g, N_HP, N_LP)
        hp += [_loops_of_source(first + j, True) for j in range(N_HP)]
        lphp += [_loops_of_source(first + j, False) for j in range(N_HP)]
        lp += [_loops_of_source(first + j, False) for j in range(N_HP, n)]
    np.testing.assert_array_equal(got["hp"], np.stack(hp))
    np.testing.assert_array_equal(got["lphp"], np.stack(lphp))
    np.testing.assert_array_equal(got["lp"], np.stack(lp))
    from oracle import tsm as otsm
    c = lambda a: a.view(np.complex128)
    m1 = otsm.tsm_combine(c(got["hp"]), c(got["lphp"]), c(got["lp"]))
    m2 = otsm.tsm_combine(c(np.stack(hp)), c(np.stack(lphp)), c(np.stack(lp)))
    for a, b in zip(m1, m2):
        np.testing.assert_array_equal(a, b)


def _hold_lock(i, q):
    import time
    from paper_1401_6749_gb300 import build
    with build.build_lock():
        q.put(("in", i, time.monotonic()))
        time.sleep(0.3)
        q.put(("out", i, time.monotonic()))


def test_build_lock_is_exclusive():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_hold_lock, args=(i, q)) for i in range(3)]
    for p in ps:
        p.start()
    ev = sorted((q.get(timeout=60) for _ in range(6)), key=lambda e: e[2])
    for p in ps:
        p.join()
    # strictly alternating in/out of the same process: no two holders at once
    for k in range(0, 6, 2):
        assert ev[k][0] == "in" and ev[k + 1][0] == "out" and ev[k][1] == ev[k + 1][1]
