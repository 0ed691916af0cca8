"""GPU tests of the services around the kernels: the context's cancel flag,
resumable runs (segments with the flag tested between them), cancelling
server jobs, the server's per-job JSON lines, and the autotune cache.

Cancellation is a host flag: no kernel is interrupted, so nothing here can
fault or hang a GPU; a resumed run must give the bits of one uninterrupted
jarzynski_run_ex call."""
import json
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

import paper_2304_03311_gb300 as jz  # noqa: E402
from paper_2304_03311_gb300 import build as jzbuild  # noqa: E402
from paper_2304_03311_gb300 import workloads as wl  # noqa: E402

JOB = wl.Job(2, 32, 32, wl.BETA_C_2D, 9, 40, 1, 96, seed=21, n_therm=30)


def _params(j):
    return jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                          n_therm=j.n_therm, direction=j.direction, traj0=j.traj0,
                          update=j.update)


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


def _reference(ctx, job):
    w = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
    s = torch.empty(job.n_traj * job.sites, dtype=torch.int8, device="cuda")
    jz.jarzynski_run_ex(ctx, _params(job), w, s)
    jz.ising_sync(ctx)
    return w.cpu().numpy(), s.cpu().numpy()


def _buffers(job):
    return (torch.zeros(job.n_traj, dtype=torch.int64, device="cuda"),
            torch.zeros(job.n_traj * job.sites, dtype=torch.int8, device="cuda"))


def test_cancel_flag_refuses_new_work_until_reset(ctx):
    w = torch.empty(JOB.n_traj, dtype=torch.int64, device="cuda")
    jz.ising_cancel(ctx)
    try:
        for call in (lambda: jz.jarzynski_run_ex(ctx, _params(JOB), w),
                     lambda: jz.jarzynski_run_batch(ctx, [_params(JOB)], [w]),
                     lambda: jz.jarzynski_run_plain(ctx, _params(JOB.with_(n_traj=2)), w),
                     lambda: jz.ising_autotune(ctx, _params(JOB))):
            with pytest.raises(jz.IsingError) as e:
                call()
            assert e.value.code == jz.ISING_ERR_CANCELLED
    finally:
        jz.ising_cancel_reset(ctx)
    jz.jarzynski_run_ex(ctx, _params(JOB), w)
    jz.ising_sync(ctx)


@pytest.mark.parametrize("update", [0, 1])
def test_resumable_run_stops_and_resumes_to_the_same_bits(ctx, update):
    job = JOB.with_(update=update)
    W_ref, S_ref = _reference(ctx, job)
    w, s = _buffers(job)
    p = _params(job)
    rc, k = jz.jarzynski_run_resumable(ctx, p, 7, w, s, k_done=0, max_segments=2)
    assert rc == jz.ISING_ERR_PENDING and k == 14
    rc, k = jz.jarzynski_run_resumable(ctx, p, 5, w, s, k_done=k, max_segments=1)
    assert rc == jz.ISING_ERR_PENDING and k == 19
    rc, k = jz.jarzynski_run_resumable(ctx, p, 9, w, s, k_done=k)
    assert rc == jz.ISING_OK and k == job.n_step
    np.testing.assert_array_equal(w.cpu().numpy(), W_ref)
    np.testing.assert_array_equal(s.cpu().numpy(), S_ref)


def test_resumable_run_cancelled_before_and_during(ctx):
    W_ref, S_ref = _reference(ctx, JOB)
    w, s = _buffers(JOB)
    p = _params(JOB)
    jz.ising_cancel(ctx)
    rc, k = jz.jarzynski_run_resumable(ctx, p, 4, w, s, k_done=0)
    jz.ising_cancel_reset(ctx)
    assert rc == jz.ISING_ERR_CANCELLED and k == 0
    # cancel from another host thread while segments run: the run stops at a
    # segment boundary (or finishes first); resuming gives the same bits
    long_job = JOB.with_(n_step=400, n_traj=2048)
    W_long, S_long = _reference(ctx, long_job)
    w2, s2 = _buffers(long_job)
    p2 = _params(long_job)
    out = {}

    def runner():
        out["r"] = jz.jarzynski_run_resumable(ctx, p2, 10, w2, s2, k_done=0)

    th = threading.Thread(target=runner)
    th.start()
    time.sleep(0.05)
    jz.ising_cancel(ctx)
    th.join(120)
    jz.ising_cancel_reset(ctx)
    rc, k = out["r"]
    assert rc in (jz.ISING_ERR_CANCELLED, jz.ISING_OK)
    assert k % 10 == 0 and 0 <= k <= long_job.n_step
    if rc == jz.ISING_ERR_CANCELLED:
        rc, k = jz.jarzynski_run_resumable(ctx, p2, 10, w2, s2, k_done=k)
    assert rc == jz.ISING_OK and k == long_job.n_step
    np.testing.assert_array_equal(w2.cpu().numpy(), W_long)
    np.testing.assert_array_equal(s2.cpu().numpy(), S_long)


def test_server_cancels_queued_and_running_jobs_and_logs_lines(ctx, tmp_path):
    log = tmp_path / "jobs.jsonl"
    server = jz.jz_server_create(ctx, 1 << 30, 1)          # one slot: later jobs queue
    try:
        jz.jz_server_set_log(server, log)
        long_job = JOB.with_(n_step=3000, n_traj=16384, seed=1)
        short = [JOB.with_(seed=2 + i) for i in range(3)]
        first = jz.jz_submit(server, _params(long_job))
        queued = [jz.jz_submit(server, _params(j)) for j in short]
        time.sleep(0.05)
        jz.jz_cancel(server, queued[1])                     # still queued: dropped
        jz.jz_cancel(server, first)                         # on the device: discarded
        res = {i: jz.jz_wait(server, i, 600.0) for i in [first] + queued}
        assert res[queued[1]].status == jz.ISING_ERR_CANCELLED
        assert res[first].status in (jz.ISING_ERR_CANCELLED, jz.ISING_OK)
        for i in (queued[0], queued[2]):
            assert res[i].status == jz.ISING_OK
        done = jz.jz_wait(server, queued[0], 1.0)
        jz.jz_cancel(server, queued[0])                     # finished: keeps its result
        assert jz.jz_wait(server, queued[0], 1.0).status == jz.ISING_OK
        assert done.delta_S2 == jz.jz_wait(server, queued[0], 1.0).delta_S2
        with pytest.raises(jz.IsingError) as e:
            jz.jz_cancel(server, 10**9)
        assert e.value.code == jz.ISING_ERR_NOT_FOUND
    finally:
        jz.jz_server_free(server)
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert sorted(d["job"] for d in lines) == sorted([first] + queued)
    by_id = {d["job"]: d for d in lines}
    assert by_id[queued[1]]["status"] == jz.ISING_ERR_CANCELLED
    ok = by_id[queued[0]]
    assert ok["status"] == 0 and ok["delta_S2"] == pytest.approx(res[queued[0]].delta_S2, rel=0,
                                                                 abs=0)
    assert ok["latency_s"] >= 0 and ok["spin_updates"] == JOB.updates


def test_server_free_finishes_queued_jobs_as_cancelled(ctx):
    server = jz.jz_server_create(ctx, 1 << 30, 1)
    ids = [jz.jz_submit(server, _params(JOB.with_(n_step=3000, n_traj=8192, seed=s)))
           for s in range(4)]
    results = {}

    def waiter(i):
        results[i] = jz.jz_wait(server, i, 600.0)

    threads = [threading.Thread(target=waiter, args=(i,)) for i in ids[1:]]
    for t in threads:
        t.start()
    time.sleep(0.02)
    jz.jz_server_free(server)
    for t in threads:
        t.join(60)
    # every waiter returned: each queued job either ran or was dropped as cancelled
    assert set(results) == set(ids[1:])
    assert all(r.status in (jz.ISING_OK, jz.ISING_ERR_CANCELLED) for r in results.values())


def test_autotune_cache_hit_skips_timing(ctx, tmp_path):
    cache = jz.TuneCache()
    p = _params(JOB.with_(n_traj=4096))
    t1, hit1 = jz.ising_autotune_cached(ctx, cache, p)
    assert not hit1 and len(cache) == 1
    t2, hit2 = jz.ising_autotune_cached(ctx, cache, p)
    assert hit2 and t2 == t1
    path = tmp_path / "tune.json"
    cache.save(path)
    other = jz.TuneCache()
    other.load(path)
    t3, hit3 = jz.ising_autotune_cached(ctx, other, p)
    assert hit3 and t3 == t1
    # the cached size is the context's size for that shape: results unchanged
    w = torch.empty(p.n_traj, dtype=torch.int64, device="cuda")
    jz.jarzynski_run_ex(ctx, p, w)
    jz.ising_sync(ctx)
