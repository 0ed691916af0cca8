"""GPU parity of the Swendsen-Wang update (update = 1) against the CPU oracle.

Bit-exact: W_int per trajectory and the final spins.  The cluster partition of
a sweep is unique, and so is its smallest site index, the root whose bit in
the sweep's flip stream decides the cluster's flip; so the concurrent union-find of the GPU and
the sequential one of the oracle must give the same configuration after every
sweep.  Cases span several warps of sites and ragged tails (V not a multiple of
32), both directions, 2D and 3D, l = 0 and l = L-1, beta = 0 (no bonds) and a
deep ordered phase (one big cluster), L_t = 2 and L = 2, several sweeps per
step, large traj0 and seeds; the full 2D L = 64 scan workload is checked on
trajectories sampled from one batched launch.  The allocation-free entry
point and persistent plans (alone and mixed with Metropolis jobs) give the
same bits.
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

BC2, BC3 = wl.BETA_C_2D, wl.BETA_C_3D
SW = jz.SWENDSEN_WANG


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


def params(job):
    return jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                          job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                          traj0=job.traj0, update=SW)


def gpu_run(ctx, job, on_device=True):
    dev = "cuda" if on_device else "cpu"
    w = torch.empty(job.n_traj, dtype=torch.int64, device=dev)
    s = torch.empty(job.n_traj * job.sites, dtype=torch.int8, device=dev)
    jz.jarzynski_run_ex(ctx, params(job), w, s)
    jz.ising_sync(ctx)
    return w.cpu().numpy(), s.cpu().numpy().reshape(job.n_traj, -1)


def oracle_run(job, traj0=None, n_traj=None):
    W, S = oracle.run(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                      n_traj if n_traj is not None else job.n_traj, job.seed,
                      n_therm=job.n_therm, direction=job.direction,
                      traj0=job.traj0 if traj0 is None else traj0, want_spins=True, update=SW)
    return W, S.reshape(len(W), -1)


SMALL = [
    wl.Job(2, 16, 16, BC2, 4, 20, 1, 24, seed=0, n_therm=20),
    wl.Job(2, 12, 6, 0.5, 0, 7, 2, 21, seed=5, n_therm=5),              # V = 144, ragged tail
    wl.Job(2, 10, 4, 0.3, 9, 5, 1, 17, seed=6, n_therm=4, direction=-1),  # l = L-1, reverse
    wl.Job(2, 2, 2, BC2, 1, 3, 1, 50, seed=7, n_therm=3),               # V = 8
    wl.Job(2, 2, 2, BC2, 0, 4, 2, 30, seed=17, n_therm=2, direction=-1),
    wl.Job(2, 4, 2, BC2, 2, 4, 3, 21, seed=8, n_therm=2, direction=-1),  # L_t = 2
    wl.Job(2, 64, 64, BC2, 30, 6, 2, 4, seed=0, n_therm=6),
    wl.Job(2, 34, 8, 0.45, 17, 5, 1, 6, seed=9, n_therm=3),
    wl.Job(2, 256, 8, BC2, 100, 3, 1, 3, seed=10, n_therm=2),
    wl.Job(3, 4, 4, BC3, 1, 6, 1, 20, seed=11, n_therm=5),
    wl.Job(3, 6, 4, 0.25, 5, 4, 1, 9, seed=12, n_therm=3, direction=-1),  # V = 288
    wl.Job(3, 16, 8, 0.22165455, 7, 10, 1, 6, seed=13, n_therm=10),
    wl.Job(3, 2, 2, 0.3, 0, 3, 2, 40, seed=14, n_therm=2),
    wl.Job(2, 16, 16, 0.0, 4, 8, 1, 16, seed=15, n_therm=4),            # beta = 0: no bonds
    wl.Job(2, 16, 16, 2.0, 4, 8, 1, 16, seed=16, n_therm=4),            # one big cluster
    wl.Job(2, 16, 8, BC2, 3, 9, 1, 12, seed=2**64 - 1, n_therm=3, traj0=2**32 - 12),
    wl.Job(2, 8, 4, BC2, 5, 1, 1, 9, seed=3, n_therm=0),                # no thermalisation
]


@pytest.mark.parametrize("job", SMALL, ids=lambda j: f"d{j.d}L{j.L}T{j.L_t}l{j.l}dir{j.direction}")
def test_bit_exact_against_oracle(ctx, job):
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def test_host_buffers_give_the_same_result(ctx):
    job = SMALL[1]
    Wd, Sd = gpu_run(ctx, job, on_device=True)
    Wh, Sh = gpu_run(ctx, job, on_device=False)
    np.testing.assert_array_equal(Wd, Wh)
    np.testing.assert_array_equal(Sd, Sh)


def test_batch_mixes_updates_and_shapes(ctx):
    jobs = [SMALL[0], SMALL[0].with_(l=7), SMALL[9], SMALL[1]]
    kinds = [SW, 0, SW, SW]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    ps = [jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                         n_therm=j.n_therm, direction=j.direction, update=u)
          for j, u in zip(jobs, kinds)]
    jz.jarzynski_run_batch(ctx, ps, outs)
    jz.ising_sync(ctx)
    for j, u, o in zip(jobs, kinds, outs):
        W, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                          n_therm=j.n_therm, direction=j.direction, update=u)
        np.testing.assert_array_equal(o.cpu().numpy(), W)


def test_range_split_matches_one_launch(ctx):
    job = SMALL[0]
    W, S = gpu_run(ctx, job)
    part = job.with_(traj0=10, n_traj=9)
    Wp, Sp = gpu_run(ctx, part)
    np.testing.assert_array_equal(Wp, W[10:19])
    np.testing.assert_array_equal(Sp, S[10:19])


def test_full_scan_workload_sampled(ctx):
    """The 2D L = 64, L_t = 64 c-function scan with the Swendsen-Wang update, as
    the benchmark's cluster mode launches it (all 31 transformations in one
    batched call), checked on sampled trajectories of three of them."""
    jobs = [j.with_(n_traj=256, update=SW) for j in wl.config2_sw().jobs]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    jz.jarzynski_run_batch(ctx, [params(j) for j in jobs], outs)
    jz.ising_sync(ctx)
    for jl in (0, 15, 30):
        job = jobs[jl]
        got = outs[jl].cpu().numpy()
        for t in (0, 255):
            W, _ = oracle_run(job, traj0=job.traj0 + t, n_traj=1)
            assert got[t] == W[0], (jl, t)


def test_server_runs_the_cluster_update(ctx):
    jobs = [SMALL[0], SMALL[9], SMALL[1]]
    server = jz.jz_server_create(ctx, 1 << 30, 2)
    try:
        ids = [jz.jz_submit(server, params(j)) for j in jobs]
        for jid, j in zip(ids, jobs):
            assert jz.jz_wait(server, jid, 600.0).status == 0
            W = np.empty(j.n_traj, dtype=np.int64)
            jz.jz_server_work(server, jid, W)
            np.testing.assert_array_equal(W, oracle_run(j)[0])
    finally:
        jz.jz_server_free(server)


def test_plain_baseline_refuses_the_cluster_update(ctx):
    job = SMALL[0]
    w = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_plain(ctx, params(job), w)
    assert e.value.code == jz.ISING_ERR_UNSUPPORTED


def test_autotune_reports_the_fixed_cta(ctx):
    assert jz.ising_autotune(ctx, params(SMALL[0])) == 256
    assert jz.ising_autotune(ctx, params(SMALL[9])) == 512


@pytest.mark.parametrize("k", [0, 1, 2, 6, 10, 13])
def test_noalloc_equals_the_oracle(k):
    job = SMALL[k]
    w = torch.full((job.n_traj,), -7, dtype=torch.int64, device="cuda")
    jz.jarzynski_run_noalloc(params(job), w)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(w.cpu().numpy(), oracle_run(job)[0])


def test_noalloc_refuses_hbm_lattices():
    job = wl.Job(2, 64, 512, BC2, 20, 2, 1, 4, seed=31, n_therm=2)   # beyond shared memory
    w = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_noalloc(params(job), w)
    assert e.value.code == jz.ISING_ERR_UNSUPPORTED


@pytest.mark.parametrize("cta", [256, 0])
def test_plan_with_cluster_and_metropolis_jobs(ctx, cta):
    """A plan mixing Swendsen-Wang jobs of three shapes with Metropolis jobs:
    one graph replay gives every job the bits of the oracle, and the batched
    estimator the oracle's Delta S_2."""
    import oracle.estimator as oest
    sw_jobs = [SMALL[i] for i in (0, 1, 6, 9, 10)]
    me_jobs = [wl.Job(2, 16, 16, BC2, 3, 12, 1, 40, seed=0, n_therm=5),
               wl.Job(3, 8, 8, BC3, 2, 10, 1, 20, seed=0, n_therm=4, direction=-1)]
    sw_jobs = [j.with_(seed=0) for j in sw_jobs]
    ps = [params(j) for j in sw_jobs]
    for j in me_jobs:
        ps.append(jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj,
                                 j.seed, n_therm=j.n_therm, direction=j.direction))
    jobs = sw_jobs + me_jobs
    outs = [torch.full((j.n_traj,), -9, dtype=torch.int64, device="cuda") for j in jobs]
    est = torch.zeros(3 * len(jobs), dtype=torch.float64, device="cuda")
    plan = jz.jz_plan_create(ctx, ps, outs, est, cta)
    try:
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    e = est.cpu().numpy().reshape(-1, 3)
    for i, (j, o) in enumerate(zip(jobs, outs)):
        W = o.cpu().numpy()
        upd = SW if i < len(sw_jobs) else 0
        ref, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                            n_therm=j.n_therm, direction=j.direction, traj0=j.traj0, update=upd)
        np.testing.assert_array_equal(W, ref)
        ref_ds, _ = oest.delta_s2_with_error(ref, j.beta, j.n_step, j.direction, 32)
        assert abs(e[i, 1] - ref_ds) <= 1e-12 * max(abs(ref_ds), 1.0)


def test_plan_of_cluster_jobs_only(ctx):
    jobs = [SMALL[i].with_(seed=0) for i in (3, 7)]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    plan = jz.jz_plan_create(ctx, [params(j) for j in jobs], outs, None, 0)
    try:
        _, _, n_items = jz.jz_plan_info(plan)
        assert n_items == 0   # no Metropolis work items
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    for j, o in zip(jobs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), oracle_run(j)[0])


@pytest.mark.parametrize("job", [
    wl.Job(2, 64, 512, BC2, 20, 2, 1, 4, seed=31, n_therm=2),            # V = 65536
    wl.Job(3, 32, 32, BC3, 9, 2, 1, 3, seed=32, n_therm=1, direction=-1),  # V = 65536
], ids=["2d_L64_T512", "3d_L32_T32"])
def test_state_beyond_shared_memory_runs_from_hbm(ctx, job):
    """Trajectories whose labels and bits exceed shared memory run from an
    HBM slice per CTA, with the bits of the oracle."""
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def test_bad_update_and_oversized_lattice_are_rejected(ctx):
    w = torch.empty(4, dtype=torch.int64, device="cuda")
    p = jz.make_params(2, 8, 8, BC2, 1, 2, 1, 4, 0, n_therm=1, update=2)
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_ex(ctx, p, w)
    assert e.value.code == jz.ISING_ERR_ARG
    # beyond shared memory the persistent plan refuses it
    p = jz.make_params(3, 32, 32, BC3, 1, 2, 1, 4, 0, n_therm=1, update=SW)
    with pytest.raises(jz.IsingError) as e:
        jz.jz_plan_create(ctx, [p], [w])
    assert e.value.code == jz.ISING_ERR_UNSUPPORTED
