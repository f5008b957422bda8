"""The multi-rank path on CPU: two gloo ranks run the host logic that a
multi-GPU job runs (sharding, slowest-rank time, job throughput, one sum of
the adjoint's parameter gradient over ranks), with the oracle standing in
for the per-rank GPU work."""
import json
import os
import socket

import numpy as np
import pytest

from paper_2510_10005_gb300 import multirank


@pytest.mark.parametrize("n", [0, 1, 7, 64, 1000003])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_partitions_cells(n, world):
    blocks = [multirank.shard(n, world, r) for r in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == n
    for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in blocks]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_shard_rejects_bad_requests():
    for args in ((10, 0, 0), (10, 2, 2), (10, 2, -1), (-1, 2, 0)):
        with pytest.raises(ValueError):
            multirank.shard(*args)


def test_single_process_fallbacks():
    assert multirank.max_over_ranks(3.5) == 3.5
    assert multirank.job_throughput(100, 1, 2, 0.5) == 400.0


OPTS = dict(method=0, reactor=1, adaptive=0, nsub=2, dt=1e-6, rtol=1e-8, atol=1e-14, newton_tol=1e-3,
            max_newton=20, max_halvings=10)
N_CELLS = 7


def _cells():
    from paper_2510_10005_gb300 import inputs
    m = inputs.gen_mechanism("h2")
    T, Y, p = inputs.field_reactor(m, N_CELLS, (1150, 1400), (1, 2), (0.5, 2.0), "H2", seed=21)
    return m, T, Y, p


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert multirank.env() == (world, rank, rank)
        m, T, Y, p = _cells()
        a, b = multirank.shard(len(T), world, rank)
        _, _, g, st = oracle.RefMech(m).adjoint_TY(T[a:b], Y[a:b], p[a:b], np.ones(b - a),
                                                   np.zeros((b - a, m.ns)), OPTS)
        dth = torch.tensor(g.sum(axis=0))                 # this rank's cells
        multirank.sum_over_ranks_(dth)
        slowest = multirank.max_over_ranks(1.0 + rank)   # rank r "took" 1 + r seconds
        multirank.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"dtheta": dth.numpy().tolist(), "slowest": slowest, "status": int(np.max(st, initial=0)),
                       "cells": b - a,
                       "throughput": multirank.job_throughput(b - a, world, 1, slowest)}, f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_sum_the_adjoint_gradient(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    m, T, Y, p = _cells()
    _, _, g, st = oracle.RefMech(m).adjoint_TY(T, Y, p, np.ones(len(T)), np.zeros_like(Y), OPTS)
    assert np.all(st == 0) and all(r["status"] == 0 for r in res)
    whole = g.sum(axis=0)
    for r in res:   # every rank holds the gradient of all cells
        np.testing.assert_allclose(np.array(r["dtheta"]), whole, rtol=1e-12, atol=1e-14 * np.abs(whole).max())
        assert r["slowest"] == 2.0
    assert sum(r["cells"] for r in res) == N_CELLS
    assert res[0]["throughput"] == world * res[0]["cells"] / 2.0
