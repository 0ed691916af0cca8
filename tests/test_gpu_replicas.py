"""GPU parity of n > 2 replicas and of the whole-cut transformation (Alba et
al., section 3) against the CPU oracle, for both updates and every entry point
that runs trajectories; and the whole-cut Renyi entropy S_n(l) against the
exact transfer matrix.

Bit-exact: W_int and the final spins of all n replicas.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.estimator as oest
import oracle.exact as ex

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

import paper_2304_03311_gb300 as jz  # noqa: E402
from paper_2304_03311_gb300 import build as jzbuild  # noqa: E402
from paper_2304_03311_gb300 import workloads as wl  # noqa: E402

BC2, BC3 = wl.BETA_C_2D, wl.BETA_C_3D


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


def params(job, update, **kw):
    return jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                          job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                          traj0=job.traj0, update=update, n_replica=job.n_replica,
                          whole=job.whole, **kw)


def gpu_run(ctx, job, update):
    w = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
    s = torch.empty(job.n_traj * job.sites, dtype=torch.int8, device="cuda")
    jz.jarzynski_run_ex(ctx, params(job, update), w, s)
    jz.ising_sync(ctx)
    return w.cpu().numpy(), s.cpu().numpy().reshape(job.n_traj, -1)


def oracle_run(job, update):
    W, S = oracle.run(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                      job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                      traj0=job.traj0, want_spins=True, update=update,
                      n_replica=job.n_replica, whole=job.whole)
    return W, S.reshape(len(W), -1)


CASES = [
    wl.Job(2, 16, 16, BC2, 4, 12, 1, 20, seed=1, n_therm=10, n_replica=3),
    wl.Job(2, 12, 6, 0.5, 0, 7, 2, 17, seed=5, n_therm=5, n_replica=3),             # ragged
    wl.Job(3, 4, 4, BC3, 1, 6, 1, 12, seed=11, n_therm=5, n_replica=3, direction=-1),
    wl.Job(2, 8, 8, BC2, 7, 5, 1, 16, seed=2, n_therm=4, n_replica=4),
    wl.Job(2, 8, 4, 0.6, 3, 4, 1, 9, seed=8, n_therm=3, n_replica=8),
    wl.Job(2, 16, 16, BC2, 8, 10, 1, 20, seed=3, n_therm=6, whole=True),            # half the row
    wl.Job(2, 16, 8, BC2, 16, 8, 1, 12, seed=4, n_therm=4, whole=True),             # the whole row
    wl.Job(2, 10, 4, 0.3, 1, 6, 2, 15, seed=6, n_therm=3, whole=True, direction=-1),
    wl.Job(2, 10, 4, 0.4, 5, 6, 1, 15, seed=7, n_therm=3, whole=True, n_replica=3),  # ragged
    wl.Job(3, 4, 4, BC3, 2, 6, 1, 10, seed=9, n_therm=4, whole=True, direction=-1),
    wl.Job(3, 6, 4, 0.25, 3, 4, 1, 8, seed=10, n_therm=3, whole=True, n_replica=3),
]


@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("job", CASES,
                         ids=lambda j: f"d{j.d}L{j.L}T{j.L_t}l{j.l}n{j.n_replica}w{int(j.whole)}")
def test_bit_exact_against_oracle(ctx, job, update):
    Wg, Sg = gpu_run(ctx, job, update)
    Wo, So = oracle_run(job, update)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def test_batch_plan_server_noalloc_agree(ctx):
    jobs = [CASES[0], CASES[5].with_(seed=1), CASES[3].with_(seed=1)]
    ref = [oracle_run(j, 0)[0] for j in jobs]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    jz.jarzynski_run_batch(ctx, [params(j, 0) for j in jobs], outs)
    jz.ising_sync(ctx)
    for o, r in zip(outs, ref):
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    pouts = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    plan = jz.jz_plan_create(ctx, [params(j, 0) for j in jobs], pouts, None, 256)
    try:
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    for o, r in zip(pouts, ref):
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    server = jz.jz_server_create(ctx, 1 << 30, 2)
    try:
        ids = [jz.jz_submit(server, params(j, 0)) for j in jobs]
        for jid, j, r in zip(ids, jobs, ref):
            assert jz.jz_wait(server, jid, 600.0).status == 0
            W = np.empty(j.n_traj, dtype=np.int64)
            jz.jz_server_work(server, jid, W)
            np.testing.assert_array_equal(W, r)
    finally:
        jz.jz_server_free(server)
    w = torch.empty(jobs[1].n_traj, dtype=torch.int64, device="cuda")
    jz.jarzynski_run_noalloc(params(jobs[1], 0), w)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(w.cpu().numpy(), ref[1])


@pytest.mark.parametrize("n", [2, 3])
def test_whole_cut_entropy_matches_transfer_matrix(ctx, n):
    """S_n(l) = -ln<e^-W>/(n-1) of the whole-cut transformation at the 2D
    critical point against the exact n-replica transfer matrix."""
    L, L_t, N = 8, 16, 200
    exact = ex.renyi_sn_transfer(2, L, L_t, BC2, n)
    jobs = [wl.Job(2, L, L_t, BC2, l, N, 1, 4096, seed=20 + l, n_therm=200, n_replica=n,
                   whole=True) for l in (1, 4, 8)]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    jz.jarzynski_run_batch(ctx, [params(j, 1) for j in jobs], outs)
    jz.ising_sync(ctx)
    for j, o in zip(jobs, outs):
        _, ds, err = jz.estimator_reduce(ctx, o, j.n_traj, j.beta, j.n_step, 1, 32)
        s_n, e_n = ds / (n - 1), err / (n - 1)
        assert abs(s_n - exact[j.l]) < 4.5 * e_n + 1e-3 * abs(exact[j.l]), (j.l, s_n, exact[j.l])


def test_bad_replica_arguments(ctx):
    w = torch.empty(4, dtype=torch.int64, device="cuda")
    base = wl.Job(2, 8, 8, BC2, 2, 4, 1, 4, n_therm=1)
    for job, code in [(base.with_(n_replica=1), jz.ISING_ERR_ARG),
                      (base.with_(n_replica=9), jz.ISING_ERR_ARG),
                      (base.with_(whole=True, l=0), jz.ISING_ERR_L_RANGE),
                      (base.with_(whole=True, l=9), jz.ISING_ERR_L_RANGE),
                      (base.with_(l=8), jz.ISING_ERR_L_RANGE)]:
        with pytest.raises(jz.IsingError) as e:
            jz.jarzynski_run_ex(ctx, params(job, 0), w)
        assert e.value.code == code
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_ex(ctx, params(base.with_(d=3, whole=True), 0, protocol=2), w)
    assert e.value.code == jz.ISING_ERR_ARG
    for job in (base.with_(n_replica=3), base.with_(whole=True)):
        with pytest.raises(jz.IsingError) as e:
            jz.jarzynski_run_plain(ctx, params(job, 0), w)
        assert e.value.code == jz.ISING_ERR_UNSUPPORTED
