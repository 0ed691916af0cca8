"""GPU parity of protocol 2 (Appendix B: the switched columns of a 3D cut move
one after another) against the CPU oracle, for both updates and every entry
point that runs trajectories.

Bit-exact: W_int (L_y times the sum of the moving column's increments) and the
final spins.  In 2D protocol 2 is protocol 1, so both must give the same bits.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

import paper_2304_03311_gb300 as jz  # noqa: E402
from paper_2304_03311_gb300 import build as jzbuild  # noqa: E402
from paper_2304_03311_gb300 import workloads as wl  # noqa: E402

BC3 = wl.BETA_C_3D


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


def params(job, update, protocol=2, **kw):
    return jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                          job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                          traj0=job.traj0, update=update, protocol=protocol, **kw)


def gpu_run(ctx, job, update, protocol=2):
    w = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
    s = torch.empty(job.n_traj * job.sites, dtype=torch.int8, device="cuda")
    jz.jarzynski_run_ex(ctx, params(job, update, protocol), w, s)
    jz.ising_sync(ctx)
    return w.cpu().numpy(), s.cpu().numpy().reshape(job.n_traj, -1)


def oracle_run(job, update, protocol=2, traj0=None, n_traj=None):
    W, S = oracle.run(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                      n_traj if n_traj is not None else job.n_traj, job.seed,
                      n_therm=job.n_therm, direction=job.direction,
                      traj0=job.traj0 if traj0 is None else traj0, want_spins=True,
                      update=update, protocol=protocol)
    return W, S.reshape(len(W), -1)


CASES = [
    wl.Job(3, 4, 4, BC3, 1, 8, 1, 20, seed=11, n_therm=5),
    wl.Job(3, 6, 4, 0.25, 5, 12, 1, 9, seed=12, n_therm=3, direction=-1),   # ragged rows
    wl.Job(3, 2, 2, 0.3, 0, 4, 2, 40, seed=14, n_therm=2),
    wl.Job(3, 16, 8, 0.22165455, 7, 32, 1, 6, seed=13, n_therm=6),
    wl.Job(3, 8, 6, 0.4, 3, 16, 2, 12, seed=15, n_therm=4, direction=-1),
]


@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("job", CASES, ids=lambda j: f"L{j.L}T{j.L_t}l{j.l}N{j.n_step}d{j.direction}")
def test_bit_exact_against_oracle(ctx, job, update):
    Wg, Sg = gpu_run(ctx, job, update)
    Wo, So = oracle_run(job, update)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)
    assert np.all(Wg % job.L == 0)          # L_y times the column's increments


@pytest.mark.parametrize("update", [0, 1])
def test_protocol2_is_protocol1_in_2d(ctx, update):
    job = wl.Job(2, 16, 8, wl.BETA_C_2D, 5, 12, 2, 17, seed=3, n_therm=4)
    W1, S1 = gpu_run(ctx, job, update, protocol=1)
    W2, S2 = gpu_run(ctx, job, update, protocol=2)
    np.testing.assert_array_equal(W1, W2)
    np.testing.assert_array_equal(S1, S2)


def test_protocols_differ_in_3d(ctx):
    job = CASES[0]
    W1, _ = gpu_run(ctx, job, 0, protocol=1)
    W2, _ = gpu_run(ctx, job, 0, protocol=2)
    assert not np.array_equal(W1, W2)


def test_slab_workload_sampled(ctx):
    """The 3D 16^3 slab scan with protocol 2 (N = 2000 = 125 steps per column),
    one batched launch, checked on sampled trajectories."""
    jobs = [j.with_(n_traj=128) for j in wl.config3().jobs]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    jz.jarzynski_run_batch(ctx, [params(j, 0) for j in jobs], outs)
    jz.ising_sync(ctx)
    for jl in (0, len(jobs) - 1):
        got = outs[jl].cpu().numpy()
        for t in (0, 127):
            W, _ = oracle_run(jobs[jl], 0, traj0=jobs[jl].traj0 + t, n_traj=1)
            assert got[t] == W[0], (jl, t)


def test_batch_plan_server_noalloc_agree(ctx):
    jobs = [CASES[0], CASES[4], CASES[0].with_(l=2)]
    ref = [oracle_run(j, 0)[0] for j in jobs]
    # one batched call mixing both protocols and updates
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    jz.jarzynski_run_batch(ctx, [params(j, 0) for j in jobs] + [params(jobs[0], 1)],
                           outs + [torch.empty(jobs[0].n_traj, dtype=torch.int64, device="cuda")])
    jz.ising_sync(ctx)
    for o, r in zip(outs, ref):
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    # persistent plan (same seed for all jobs)
    pj = [j.with_(seed=5) for j in jobs]
    pref = [oracle_run(j, 0)[0] for j in pj]
    pouts = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in pj]
    plan = jz.jz_plan_create(ctx, [params(j, 0) for j in pj], pouts, None, 256)
    try:
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    for o, r in zip(pouts, pref):
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    # server
    server = jz.jz_server_create(ctx, 1 << 30, 2)
    try:
        ids = [jz.jz_submit(server, params(j, 0)) for j in jobs]
        for jid, j, r in zip(ids, jobs, ref):
            res = jz.jz_wait(server, jid, 600.0)
            assert res.status == 0
            W = np.empty(j.n_traj, dtype=np.int64)
            jz.jz_server_work(server, jid, W)
            np.testing.assert_array_equal(W, r)
    finally:
        jz.jz_server_free(server)
    # allocation-free entry point
    w = torch.empty(jobs[1].n_traj, dtype=torch.int64, device="cuda")
    jz.jarzynski_run_noalloc(params(jobs[1], 0), w)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(w.cpu().numpy(), ref[1])


def test_bad_protocol_arguments(ctx):
    w = torch.empty(4, dtype=torch.int64, device="cuda")
    job = wl.Job(3, 4, 4, BC3, 1, 6, 1, 4, n_therm=1)        # 6 steps, 4 columns
    for p, code in [(params(job, 0), jz.ISING_ERR_ARG),
                    (params(job.with_(n_step=8), 0, protocol=3), jz.ISING_ERR_ARG)]:
        with pytest.raises(jz.IsingError) as e:
            jz.jarzynski_run_ex(ctx, p, w)
        assert e.value.code == code
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_plain(ctx, params(job.with_(n_step=8), 0), w)
    assert e.value.code == jz.ISING_ERR_UNSUPPORTED
