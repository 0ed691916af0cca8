"""Multi-rank host logic on CPU (gloo, world size 2): sharded trajectories
gathered over the process group equal the one-shot run bit for bit, and a rank
that dies before the exchange is reported as a missing shard, not a hang.
The per-rank work is produced by the CPU oracle (no GPU involved)."""
import datetime
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import oracle.estimator as oest  # noqa: E402
from paper_2304_03311_gb300 import shard  # noqa: E402

JOB = dict(d=2, L=8, L_t=8, beta=0.44068679350977147, l=3, n_step=12, n_sweep=1, seed=5)
N_TRAJ = 37


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir, die_rank):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    first, count = shard.shard_range(N_TRAJ, rank, world)
    W, _ = oracle.run(JOB["d"], JOB["L"], JOB["L_t"], JOB["beta"], JOB["l"], JOB["n_step"],
                      JOB["n_sweep"], count, JOB["seed"], n_therm=20, traj0=first)
    if rank == die_rank:
        os._exit(0)            # leaves between steps, nothing in flight
    result = {}
    try:
        merged = shard.gather_work(W, N_TRAJ)
        result["merged"] = merged.tolist()
    except shard.MissingShardError as exc:
        result["missing"] = str(exc)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(result, f)
    if "missing" not in result:
        dist.destroy_process_group()


def _run(world, die_rank, tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path), die_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank hung")
    out = {}
    for r in range(world):
        path = tmp_path / f"rank{r}.json"
        if path.exists():
            out[r] = json.loads(path.read_text())
    return out


def test_shard_ranges_cover_once():
    for n in (0, 1, 7, 37, 1000):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_range(n, r, world, traj0=11) for r in range(world)]
            idx = [i for a, c in spans for i in range(a, a + c)]
            assert idx == list(range(11, 11 + n))


def test_merge_rejects_missing_or_short_shards():
    parts = {0: np.arange(19), 1: np.arange(18)}
    assert shard.merge_shards(parts, 37, 2).size == 37
    with pytest.raises(shard.MissingShardError):
        shard.merge_shards({0: np.arange(19)}, 37, 2)
    with pytest.raises(shard.MissingShardError):
        shard.merge_shards({0: np.arange(19), 1: np.arange(17)}, 37, 2)


def test_two_ranks_gather_equals_one_shot(tmp_path):
    out = _run(2, -1, tmp_path)
    W1, _ = oracle.run(JOB["d"], JOB["L"], JOB["L_t"], JOB["beta"], JOB["l"], JOB["n_step"],
                       JOB["n_sweep"], N_TRAJ, JOB["seed"], n_therm=20)
    for r in (0, 1):
        merged = np.array(out[r]["merged"], dtype=np.int64)
        np.testing.assert_array_equal(merged, W1)
    # the estimator over the gathered array is the single-process estimator
    a = oest.delta_s2_with_error(np.array(out[0]["merged"]), JOB["beta"], JOB["n_step"])
    b = oest.delta_s2_with_error(W1, JOB["beta"], JOB["n_step"])
    assert a == b


def test_dead_rank_is_reported_missing(tmp_path):
    out = _run(2, 1, tmp_path)
    assert 1 not in out
    assert "missing" in out[0]


def _bench_worker(rank, world, port, out_dir, die_rank):
    """The benchmark's own exchange (bench.exchange_work) on its weak-scaling
    layout: rank r runs trajectories [r n, (r+1) n) of every l; stand-in work
    values encode (global trajectory, l) so the gathered order is checkable."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    w = bench.workload_for(2, rank, traj_per_l=5)
    arrays = [np.arange(j.traj0, j.traj0 + j.n_traj, dtype=np.int64) * 1000 + j.l for j in w.jobs]
    if rank == die_rank:
        os._exit(0)
    result = {}
    try:
        merged = bench.exchange_work(arrays, w.jobs, world, None)
        result["merged"] = [m.tolist() for m in merged]
    except shard.MissingShardError as exc:
        result["missing"] = str(exc)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(result, f)
    if "missing" not in result:
        dist.destroy_process_group()


def _run_bench(world, die_rank, tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, world, port, str(tmp_path), die_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank hung")
    return {r: json.loads((tmp_path / f"rank{r}.json").read_text())
            for r in range(world) if (tmp_path / f"rank{r}.json").exists()}


def test_bench_exchange_gathers_every_l_in_global_order(tmp_path):
    out = _run_bench(2, -1, tmp_path)
    for r in (0, 1):
        merged = out[r]["merged"]
        assert len(merged) == 31
        for l, m in enumerate(merged):
            assert m == [t * 1000 + l for t in range(10)]


def test_bench_exchange_reports_a_dead_rank(tmp_path):
    out = _run_bench(2, 1, tmp_path)
    assert 1 not in out
    assert "missing" in out[0]
