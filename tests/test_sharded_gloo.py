"""Multi-rank path sharding on CPU: world_size 2 and 3 over gloo (no GPU).

The per-rank sums come from a stand-in that sums the FP64 oracle's per-path
payoffs over the rank's path range (the CUDA path_sums needs a GPU); what is
tested is the host-side logic: the shard ranges cover [0, P) exactly once, the
all-reduce combines them, the combined sums equal the single-process sums, and a
rank that fails on the host (an exception before the exchange) ends the other
ranks' all-reduce with an error within the group's timeout instead of a hang.
"""
import datetime
import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads
from paper_2402_12111_gb300.sharded import shard_range, sharded_sums

MODEL = dict(workloads.BASE_MODEL)
K = np.array([90.0, 100.0, 110.0])
STEPS, PATHS, SEED = 16, 5003, 21


def oracle_sums(model, strikes, is_put, steps, begin, count, seed=1, greeks=(), rel_bump=1e-4, option_index=0):
    x, _, _ = oracle.terminal(model, steps, seed, begin, count, option_index=option_index)
    S = model["S0"] * np.exp(x)
    f = np.maximum(S[None, :] - np.asarray(strikes)[:, None], 0.0)
    return torch.tensor(np.stack([f.sum(axis=1), (f * f).sum(axis=1)], axis=1), dtype=torch.float64)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = sharded_sums(MODEL, K, False, STEPS, PATHS, SEED, sums_fn=oracle_sums)
    torch.save(s, os.path.join(out_dir, f"r{rank}.pt"))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sums_equal_whole(world, tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    whole = oracle_sums(MODEL, K, False, STEPS, 0, PATHS, seed=SEED)
    for r in range(world):
        s = torch.load(os.path.join(tmp_path, f"r{r}.pt"))
        torch.testing.assert_close(s, whole, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("paths,world", [(10, 3), (5003, 2), (1, 4), (1 << 20, 8), (7, 7)])
def test_shard_ranges_partition(paths, world):
    seen = []
    for r in range(world):
        b, n = shard_range(paths, r, world)
        seen.extend(range(b, b + n))
    assert seen == list(range(paths))
    with pytest.raises(ValueError):
        shard_range(paths, world, world)


def _failing_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))

    def sums(*args, **kwargs):
        if rank == world - 1:
            raise RuntimeError("planted host-side failure")
        return oracle_sums(*args, **kwargs)

    t0 = time.monotonic()
    try:
        sharded_sums(MODEL, K, False, STEPS, PATHS, SEED, sums_fn=sums)
        status = "ok"
    except Exception as e:  # the failed rank's own error, or the collective's on the others
        status = f"error {type(e).__name__}: {e}"
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{time.monotonic() - t0:.3f}\n{status}")
    # the failed rank leaves between steps, with no collective in flight; the
    # others learn of it from their collective, which ends with an error


@pytest.mark.parametrize("world", [2, 3])
def test_a_failed_rank_ends_the_others_collective_with_an_error(world, tmp_path):
    port = _free_port()
    mp.start_processes(_failing_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        with open(os.path.join(tmp_path, f"r{r}.txt")) as f:
            elapsed, status = f.read().split("\n", 1)
        assert status.startswith("error"), (r, status)
        if r == world - 1:
            assert "planted host-side failure" in status
        else:
            # the surviving ranks do not hang: the collective fails within the group's timeout
            assert float(elapsed) < 30.0, (r, elapsed, status)
