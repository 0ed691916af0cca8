"""GPU tests of the continuous-batching server (jz_server_* / jz_submit).

Each job's result -- W_int of every trajectory and the estimator values --
must be the same whether the job runs alone or in a mix of jobs that arrive
together, arrive while others run, or wait for device memory; jobs that fit
together must overlap on the device; admission, timeouts and unknown ids
report their error codes.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

import paper_2304_03311_gb300 as jz  # noqa: E402
from paper_2304_03311_gb300 import build as jzbuild  # noqa: E402
from paper_2304_03311_gb300 import workloads as wl  # noqa: E402


def _params(j):
    return jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                          n_therm=j.n_therm, direction=j.direction, traj0=j.traj0)


def _need(j):
    tcut = j.n_step * 8 * j.d * 4
    return ((tcut + 255) & ~255) + 256 + 8 * j.n_traj + 256


def _mix():
    out = []
    for i, (d, L, Lt) in enumerate([(2, 32, 32), (3, 8, 8), (2, 48, 48), (3, 12, 12),
                                    (2, 16, 16), (2, 34, 34), (3, 16, 16), (2, 64, 64)]):
        beta = (wl.BETA_C_2D if d == 2 else wl.BETA_C_3D) * (0.9, 1.0, 1.1)[i % 3]
        out.append(wl.Job(d, L, Lt, beta, 1 + (i * 5) % (L // 2), 40 + 10 * i, 1, 64 + 32 * i,
                          seed=100 + i, n_therm=50, direction=1 if i % 4 else -1))
    return out


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


@pytest.fixture(scope="module")
def alone(ctx):
    res = {}
    for j in _mix():
        w = torch.empty(j.n_traj, dtype=torch.int64, device="cuda")
        jz.jarzynski_run_ex(ctx, _params(j), w)
        jz.ising_sync(ctx)
        est = jz.estimator_reduce(ctx, w, j.n_traj, j.beta, j.n_step, j.direction, 32)
        res[j] = (w.cpu().numpy(), est)
    return res


def _check(server, jid, j, alone):
    r = jz.jz_wait(server, jid, 600.0)
    assert r.status == jz.ISING_OK
    W = np.empty(j.n_traj, dtype=np.int64)
    jz.jz_server_work(server, jid, W)
    W_ref, (lr, ds, err) = alone[j]
    np.testing.assert_array_equal(W, W_ref)
    assert (r.log_ratio, r.delta_S2, r.delta_S2_err) == (lr, ds, err)
    assert r.updates == j.updates
    assert r.submit_s <= r.start_s <= r.done_s
    return r


def test_mix_arriving_together_equals_alone(ctx, alone):
    server = jz.jz_server_create(ctx, 1 << 30, 4)
    try:
        jobs = _mix()
        ids = [jz.jz_submit(server, _params(j)) for j in jobs]
        rs = [_check(server, i, j, alone) for i, j in zip(ids, jobs)]
    finally:
        jz.jz_server_free(server)
    # four slots: some jobs ran at the same time
    overlaps = sum(1 for a in rs for b in rs if a is not b and a.start_s < b.start_s < a.done_s)
    assert overlaps >= 1


def test_staggered_arrivals_equal_alone(ctx, alone):
    server = jz.jz_server_create(ctx, 1 << 30, 3)
    try:
        jobs = _mix()
        ids = []
        for j in jobs:
            ids.append(jz.jz_submit(server, _params(j)))
            time.sleep(0.002)
        for i, j in zip(ids, jobs):
            _check(server, i, j, alone)
    finally:
        jz.jz_server_free(server)


def test_budget_bounds_what_runs_together(ctx, alone):
    jobs = _mix()
    budget = max(_need(j) for j in jobs)
    server = jz.jz_server_create(ctx, budget, 8)
    try:
        ids = [jz.jz_submit(server, _params(j)) for j in jobs]
        rs = [_check(server, i, j, alone) for i, j in zip(ids, jobs)]
        # admitted in arrival order
        starts = [r.start_s for r in rs]
        assert starts == sorted(starts)
        # the jobs on the device at any start time fit the budget together
        for r in rs:
            running = [_need(j) for j, o in zip(jobs, rs) if o.start_s <= r.start_s < o.done_s]
            assert sum(running) <= budget
        too_big = jobs[-1].with_(n_traj=budget // 8 + 1)
        jid = jz.jz_submit(server, _params(too_big))
        assert jz.jz_wait(server, jid, 60.0).status == jz.ISING_ERR_NOMEM
    finally:
        jz.jz_server_free(server)


def test_timeout_unknown_and_invalid(ctx):
    server = jz.jz_server_create(ctx, 1 << 30, 1)
    try:
        long_job = wl.Job(2, 64, 64, wl.BETA_C_2D, 10, 4000, 2, 4096, seed=3)
        jid = jz.jz_submit(server, _params(long_job))
        with pytest.raises(jz.IsingError) as e:
            jz.jz_wait(server, jid, 0.0)
        assert e.value.code == jz.ISING_ERR_TIMEOUT
        assert jz.jz_poll(server, jid) is None
        with pytest.raises(jz.IsingError) as e:
            jz.jz_poll(server, 987654321)
        assert e.value.code == jz.ISING_ERR_NOT_FOUND
        with pytest.raises(jz.IsingError) as e:
            jz.jz_submit(server, jz.make_params(2, 7, 8, 0.4, 1, 5, 1, 4, 0))
        assert e.value.code == jz.ISING_ERR_ODD_EXTENT
    finally:
        jz.jz_server_free(server)     # waits for the long job, drops nothing queued


def test_alone_reference_matches_oracle(alone):
    """The mix's "alone" results (each job run by itself through
    jarzynski_run_ex) are the oracle's bits, so the mix-invariance tests
    compare the server against the oracle too."""
    import oracle
    for j in _mix():
        Wo, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                           n_therm=j.n_therm, direction=j.direction, traj0=j.traj0)
        np.testing.assert_array_equal(alone[j][0], Wo)
