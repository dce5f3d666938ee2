"""Particle sharding across ranks on CPU (gloo, world sizes 2 and 3): the gathered weights equal
the single-rank array on every rank, every rank computes the same ancestors, and after the row
exchange the shards' particles concatenate to the single-rank resampling result -- bit for bit on
dyadic weights (Sec. 2.4: systematic resampling; Sec. 3.4: the increment needs all J weights)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import smc as osmc  # noqa: E402
from paper_1709_09763_gb300 import sharded  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem(J, K, seed):
    rng = np.random.default_rng(seed)
    logw = np.log(2.0 ** rng.integers(-10, 0, size=J))          # dyadic weights
    theta = rng.normal(0, 1, (J, K))
    phi = rng.uniform(0, 50, J)
    return logw, theta, phi


def _worker(rank, world, port, J, K, U, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    logw, theta, phi = _problem(J, K, 11)
    bounds = sharded.shard_bounds(J, world)
    lo, hi = bounds[rank]
    # 1) all-gather of the local log-weights: identical full arrays on every rank
    full = sharded.allgather_rows(torch.from_numpy(logw[lo:hi]).clone()).numpy()
    # 2) every rank computes the same ancestors from the gathered weights
    anc = osmc.systematic_resample(full, U)
    # 3) rows move to their new owners (theta and the potential cache together)
    rows = torch.from_numpy(np.concatenate([theta[lo:hi], phi[lo:hi, None]], axis=1)).clone()
    new = sharded.exchange_rows(rows, anc, bounds).numpy()
    out.put((rank, full, anc, new))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,J", [(2, 64), (3, 37), (2, 5)])
def test_sharded_resampling_concatenates_to_single_rank_result(world, J):
    K, U = 3, 0.3141592653589793
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, J, K, U, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    logw, theta, phi = _problem(J, K, 11)
    anc_single = osmc.systematic_resample(logw, U)
    rows_single = np.concatenate([theta, phi[:, None]], axis=1)[anc_single]
    for rank, full, anc, _ in res:
        assert np.array_equal(full, logw)
        assert np.array_equal(anc, anc_single)
    got = np.concatenate([r[3] for r in res], axis=0)
    assert np.array_equal(got, rows_single)


def test_shard_bounds_and_exchange_plan():
    assert sharded.shard_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert sharded.shard_bounds(2, 4) == [(0, 1), (1, 2), (2, 2), (2, 2)]
    b = sharded.shard_bounds(8, 2)
    anc = np.array([0, 0, 1, 5, 5, 6, 7, 7])
    plan = sharded.exchange_plan(anc, b)
    # rank 0's outputs 0..3 take 0, 0, 1 from itself and 5 from rank 1; rank 1's all from rank 1
    assert plan[0] == {0: (0, 3)}
    assert plan[1] == {0: (3, 1), 1: (0, 4)}
    assert list(sharded.owner_of([0, 3, 4, 7], b)) == [0, 0, 1, 1]
    with pytest.raises(ValueError):
        sharded.exchange_plan(np.array([1, 0, 2, 3, 4, 5, 6, 7]), b)
    with pytest.raises(ValueError):
        sharded.owner_of([8], b)
