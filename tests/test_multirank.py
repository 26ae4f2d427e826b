"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs its own replica, the slowest rank's time decides, and the whole-job
value counts every rank's iterations."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_timing(local_ms[rank], 100, world, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank():
    world, port = 2, _free_port()
    local_ms = [3.0, 5.0]  # rank 1 is slower
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, local_ms, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == pytest.approx(5.0 / 100)
        assert value == pytest.approx(2 * 100 / 5e-3)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_timing(7.0, 70, 1, torch.device("cpu"))
    assert ms == pytest.approx(0.1) and value == pytest.approx(10_000.0)


def _shard_worker(rank, world, port, out):
    """One CPU rank of a row-sharded SES iteration with the oracle standing in
    for the pass: each rank sums exp(X_i) (Sec. 2.1) over the cones of its
    rows, the ranks exchange one row each with the library's exchange_rows,
    and the merged sum must give the weights of the unsharded Eq. (implement)."""
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import eja, ses as oses
    from paper_2405_09157_gb300 import api, datagen
    n, d = 101, 3
    V = datagen.ses_gaussian(n, d, seed=5).astype(np.float64)
    ubar, alpha, k = V[0] + 0.25, 2.0, 0.7
    lo, hi = api.shard_rows(n, world, rank)
    X = oses.ses_exponent(V, None, ubar, alpha, k)       # rows of cones 2..n (input rows 1..n-1)
    mine = X[max(lo, 1) - 1:hi - 1]                       # rank 0 skips row 0, the easy cone
    row = torch.tensor(np.concatenate([eja.soc_exp(mine).sum(axis=0), [float(rank), hi - lo]]))
    rows = api.exchange_rows(row, world)
    out[rank] = (rows.numpy().copy(), lo, hi)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_sharded_exchange_merges_in_rank_order(world):
    import numpy as np
    from oracle import eja, ses as oses
    from paper_2405_09157_gb300 import api, datagen
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    n, d = 101, 3
    spans = [out[r][1:] for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n                      # the shards cover the rows once
    assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
    assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    for r in range(world):
        rows = out[r][0]
        assert rows.shape == (world, d + 3)
        assert np.array_equal(rows, out[0][0])                           # every rank sees the same rows
        assert np.array_equal(rows[:, d + 1], np.arange(world))          # in rank order
    merged = out[0][0][:, :d + 1].sum(axis=0)
    V = datagen.ses_gaussian(n, d, seed=5).astype(np.float64)
    P = oses.ses_weights(V, None, V[0] + 0.25, 2.0, 0.7)
    assert np.allclose(P.sum(axis=0), merged / eja.soc_trace(merged), rtol=1e-12, atol=1e-15)


def test_shard_rows_split():
    from paper_2405_09157_gb300 import api
    assert [api.shard_rows(10, 3, r) for r in range(3)] == [(0, 4), (4, 7), (7, 10)]
    assert api.shard_rows(5, 1, 0) == (0, 5)
    with pytest.raises(ValueError):
        api.shard_rows(2, 3, 0)
