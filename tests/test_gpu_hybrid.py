"""GPU parity of the Swendsen-Wang thermalisation option (therm_update = 1):
a thermalisation-only sw_kernel launch, then the Metropolis protocol from its
spins, against the oracle's single trajectory of the same composition.

Bit-exact W_int and final spins on 2D and 3D shapes (ragged rows, reverse,
protocol 2, n = 3 replicas, whole cuts), inside a batch beside plain jobs, as
segments resumed mid-protocol, through the server, and with no thermalisation
sweeps (then the plain Metropolis run).  Entry points that do not serve it
refuse it.
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
H = jz.SW_THERM


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


def params(j, **kw):
    return jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep,
                          kw.get("n_traj", j.n_traj), j.seed, n_therm=j.n_therm,
                          direction=j.direction, traj0=j.traj0, protocol=j.protocol,
                          n_replica=j.n_replica, whole=j.whole,
                          therm_update=kw.get("therm_update", j.therm_update))


def oracle_run(j, therm_update=None):
    W, S = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                      n_therm=j.n_therm, direction=j.direction, traj0=j.traj0,
                      want_spins=True, protocol=j.protocol, n_replica=j.n_replica,
                      whole=j.whole,
                      therm_update=j.therm_update if therm_update is None else therm_update)
    return W, S.reshape(len(W), -1)


def gpu_run(ctx, j, **kw):
    w = torch.empty(j.n_traj, dtype=torch.int64, device="cuda")
    s = torch.empty(j.n_traj * j.sites, dtype=torch.int8, device="cuda")
    jz.jarzynski_run_ex(ctx, params(j, **kw), w, s)
    jz.ising_sync(ctx)
    return w.cpu().numpy(), s.cpu().numpy().reshape(j.n_traj, -1)


JOBS = [
    wl.Job(2, 16, 16, BC2, 4, 12, 1, 40, seed=1, n_therm=20, therm_update=H),
    wl.Job(2, 12, 6, 0.5, 0, 7, 2, 33, seed=5, n_therm=5, direction=-1, therm_update=H),
    wl.Job(2, 64, 64, BC2, 30, 5, 2, 6, seed=0, n_therm=8, therm_update=H),
    wl.Job(2, 34, 8, 0.45, 17, 5, 1, 6, seed=9, n_therm=3, therm_update=H),
    wl.Job(3, 4, 4, BC3, 1, 6, 1, 20, seed=11, n_therm=5, therm_update=H),
    wl.Job(3, 6, 4, 0.25, 5, 4, 1, 9, seed=12, n_therm=3, direction=-1, therm_update=H),
    wl.Job(3, 4, 4, BC3, 2, 8, 1, 10, seed=13, n_therm=4, protocol=2, therm_update=H),
    wl.Job(2, 8, 8, BC2, 3, 6, 1, 12, seed=14, n_therm=6, n_replica=3, therm_update=H),
    wl.Job(2, 8, 8, BC2, 3, 6, 1, 12, seed=15, n_therm=6, whole=True, therm_update=H),
    wl.Job(2, 16, 8, BC2, 3, 9, 1, 12, seed=2**64 - 1, n_therm=3, traj0=123456,
           therm_update=H),
    wl.Job(2, 6, 4, BC2, 2, 5, 1, 7, seed=16, n_therm=4, n_replica=8, therm_update=H),
    wl.Job(2, 8, 8, BC2, 5, 6, 1, 9, seed=17, n_therm=5, whole=True, direction=-1,
           therm_update=H),
]


@pytest.mark.parametrize("job", JOBS, ids=lambda j: f"d{j.d}L{j.L}Lt{j.L_t}l{j.l}n{j.n_replica}"
                         f"p{j.protocol}w{int(j.whole)}dir{j.direction}")
def test_bit_exact_with_the_oracle(ctx, job):
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def test_thermalisation_changes_the_trajectories(ctx):
    j = JOBS[0]
    Wh, Sh = gpu_run(ctx, j)
    Wm, Sm = gpu_run(ctx, j, therm_update=0)
    assert not np.array_equal(Sh, Sm)
    Wo, So = oracle_run(j, therm_update=0)
    np.testing.assert_array_equal(Sm, So)


def test_no_thermalisation_sweeps_is_the_plain_run(ctx):
    j = JOBS[0].with_(n_therm=0)
    Wh, Sh = gpu_run(ctx, j)
    Wm, Sm = gpu_run(ctx, j, therm_update=0)
    np.testing.assert_array_equal(Wh, Wm)
    np.testing.assert_array_equal(Sh, Sm)


def test_batch_mixes_the_two_starts(ctx):
    """A scan-like batch: the same l values with and without the option, one
    call; each job keeps its own bits."""
    jobs = [wl.Job(2, 16, 16, BC2, l, 10, 1, 17, seed=3, n_therm=12, therm_update=t)
            for l in (2, 5) for t in (0, H)]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    jz.jarzynski_run_batch(ctx, [params(j) for j in jobs], outs)
    jz.ising_sync(ctx)
    assert jz.ising_last_launch_ms(ctx) > 0
    for j, o in zip(jobs, outs):
        Wo, _ = oracle_run(j)
        np.testing.assert_array_equal(o.cpu().numpy(), Wo)


def test_segments_resume_to_the_one_run(ctx):
    j = JOBS[4]
    w = torch.zeros(j.n_traj, dtype=torch.int64, device="cuda")
    s = torch.zeros(j.n_traj * j.sites, dtype=torch.int8, device="cuda")
    p = params(j)
    jz.jarzynski_run_segment(ctx, p, 0, 2, w, s)
    jz.jarzynski_run_segment(ctx, p, 2, j.n_step, w, s)
    jz.ising_sync(ctx)
    Wo, So = oracle_run(j)
    np.testing.assert_array_equal(w.cpu().numpy(), Wo)
    np.testing.assert_array_equal(s.cpu().numpy().reshape(j.n_traj, -1), So)


def test_server_serves_it(ctx):
    """Jobs with and without the option through the continuous-batching
    server, concurrently: each keeps the oracle's bits."""
    jobs = [JOBS[0], JOBS[4], JOBS[0].with_(therm_update=0), JOBS[7]]
    server = jz.jz_server_create(ctx, 1 << 30, 3)
    try:
        ids = [jz.jz_submit(server, params(j)) for j in jobs]
        res = [jz.jz_wait(server, i, 600.0) for i in ids]
        assert all(r.status == 0 for r in res)
        for j, i in zip(jobs, ids):
            w = np.empty(j.n_traj, dtype=np.int64)
            jz.jz_server_work(server, i, w)
            Wo, _ = oracle_run(j)
            np.testing.assert_array_equal(w, Wo)
    finally:
        jz.jz_server_free(server)


@pytest.mark.parametrize("cta", [256, 0])
def test_persistent_plan_serves_it(ctx, cta):
    """An uneven plan of 2D and 3D jobs with and without the option (and a
    Swendsen-Wang job), replayed twice from its graph: the oracle's bits."""
    jobs = [JOBS[0], JOBS[4], JOBS[5], JOBS[0].with_(therm_update=0, traj0=1 << 20),
            wl.Job(2, 8, 8, BC2, 2, 5, 1, 9, seed=1, n_therm=4, update=1, traj0=2 << 20)]
    jobs = [j.with_(seed=1) for j in jobs]
    outs = [torch.full((j.n_traj,), -9, dtype=torch.int64, device="cuda") for j in jobs]
    ps = [params(j) for j in jobs]
    for p, j in zip(ps, jobs):
        p.update = j.update
    plan = jz.jz_plan_create(ctx, ps, outs, None, cta)
    try:
        for _ in range(2):
            for o in outs:
                o.fill_(-9)
            jz.jz_plan_launch(plan)
            jz.ising_sync(ctx)
            for j, o in zip(jobs, outs):
                W, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj,
                                  j.seed, n_therm=j.n_therm, direction=j.direction,
                                  traj0=j.traj0, update=j.update, protocol=j.protocol,
                                  therm_update=j.therm_update if j.update == 0 else None)
                np.testing.assert_array_equal(o.cpu().numpy(), W)
    finally:
        jz.jz_plan_free(plan)


def test_server_charges_the_thermalised_spins(ctx):
    """A job whose thermalised spins (n_traj V bytes) alone exceed the server's
    budget finishes with ISING_ERR_NOMEM; the same job without the option
    fits and runs."""
    j = wl.Job(2, 64, 64, BC2, 5, 4, 1, 512, seed=1, n_therm=4, therm_update=H)
    budget = 1 << 20   # 1 MiB: W_int and tables fit, 512 x 8192 bytes of spins do not
    server = jz.jz_server_create(ctx, budget, 2)
    try:
        a = jz.jz_submit(server, params(j))
        b = jz.jz_submit(server, params(j, therm_update=0))
        ra, rb = jz.jz_wait(server, a, 600.0), jz.jz_wait(server, b, 600.0)
        assert ra.status == jz.ISING_ERR_NOMEM
        assert rb.status == 0
    finally:
        jz.jz_server_free(server)


def test_full_scan_from_a_swendsen_wang_start_sampled(ctx):
    """The 2D L = 64 scan at full size (31 x 16384 trajectories, N = 1000 x 2
    sweeps) from 100 Swendsen-Wang thermalisation sweeps, one launch pair as
    `bench.py --therm-update 1 --n-therm 100` runs it with 512-thread CTAs:
    the first and last trajectory of l = 0, 15 and 30 against the oracle."""
    w = wl.config2()
    jobs = [j.with_(n_therm=100, therm_update=H) for j in w.jobs]
    c = jz.ising_replica_init(0, 0, None)
    try:
        jz.ising_set_threads(c, 2, 64, 64, 512)
        outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
        jz.jarzynski_run_batch(c, [params(j) for j in jobs], outs)
        jz.ising_sync(c)
        res = [o.cpu().numpy() for o in outs]
    finally:
        jz.ising_replica_free(c)
    for l in (0, 15, 30):
        j = jobs[l]
        assert np.all(res[l] % 2 == 0) and len(np.unique(res[l])) > 1
        for t in (0, j.n_traj - 1):
            Wo, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, 1, j.seed,
                               n_therm=j.n_therm, traj0=j.traj0 + t, therm_update=H)
            assert res[l][t] == Wo[0], (l, t)


def test_state_beyond_shared_memory_thermalises_from_hbm_in_chunks(ctx):
    """2D L = 128, L_t = 8L: its Swendsen-Wang state (1.2 MB) lives in HBM
    slices, one resident wave of trajectories per thermalisation launch; 770
    trajectories span two launches on GB300.  Trajectories on both sides of
    the chunk boundary, and the last one, keep the oracle's bits."""
    j = wl.Job(2, 128, 1024, BC2, 40, 2, 1, 770, seed=21, n_therm=2, therm_update=H)
    w = torch.empty(j.n_traj, dtype=torch.int64, device="cuda")
    jz.jarzynski_run_ex(ctx, params(j), w)
    jz.ising_sync(ctx)
    W = w.cpu().numpy()
    for t in (0, 1, 758, 759, 760, 761, 769):
        Wo, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, 1, j.seed,
                           n_therm=j.n_therm, traj0=j.traj0 + t, therm_update=H)
        assert W[t] == Wo[0], t


@pytest.mark.parametrize("how", ["batch", "plan"])
def test_waves_pack_pieces_of_several_jobs(ctx, how):
    """Three 2D L = 128, L_t = 8L jobs of 300 trajectories from a
    Swendsen-Wang start: their 900 trajectories fill the thermalisation waves
    in order (on GB300 the first wave holds all of the first two jobs and 160
    of the third), through the batch call and a plan; trajectories on every
    piece boundary keep the oracle's bits."""
    jobs = [wl.Job(2, 128, 1024, BC2, l, 2, 1, 300, seed=29, n_therm=2, therm_update=H,
                   traj0=i << 20) for i, l in enumerate((10, 40, 70))]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    if how == "batch":
        jz.jarzynski_run_batch(ctx, [params(j) for j in jobs], outs)
        jz.ising_sync(ctx)
    else:
        plan = jz.jz_plan_create(ctx, [params(j) for j in jobs], outs, None, 512)
        try:
            jz.jz_plan_launch(plan)
            jz.ising_sync(ctx)
        finally:
            jz.jz_plan_free(plan)
    for i, ts in enumerate([(0, 299), (0, 299), (0, 159, 160, 299)]):
        j = jobs[i]
        W = outs[i].cpu().numpy()
        for t in ts:
            Wo, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, 1, j.seed,
                               n_therm=j.n_therm, traj0=j.traj0 + t, therm_update=H)
            assert W[t] == Wo[0], (i, t)


def test_plan_thermalises_a_large_state_from_hbm(ctx):
    """A persistent plan with a 2D L = 128, L_t = 8L job from a Swendsen-Wang
    start (HBM thermalisation waves inside the plan's graph) beside a small
    one, replayed twice: trajectories on both sides of the chunk boundary
    keep the oracle's bits."""
    jobs = [wl.Job(2, 128, 1024, BC2, 40, 2, 1, 770, seed=21, n_therm=2, therm_update=H),
            wl.Job(2, 16, 16, BC2, 4, 6, 1, 33, seed=21, n_therm=5, therm_update=H,
                   traj0=1 << 20)]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    plan = jz.jz_plan_create(ctx, [params(j) for j in jobs], outs, None, 512)
    try:
        for _ in range(2):
            for o in outs:
                o.fill_(-9)
            jz.jz_plan_launch(plan)
            jz.ising_sync(ctx)
            W0 = outs[0].cpu().numpy()
            for t in (0, 759, 760, 769):
                Wo, _ = oracle.run(2, 128, 1024, BC2, 40, 2, 1, 1, 21, n_therm=2, traj0=t,
                                   therm_update=H)
                assert W0[t] == Wo[0], t
            Wo, _ = oracle_run(jobs[1])
            np.testing.assert_array_equal(outs[1].cpu().numpy(), Wo)
    finally:
        jz.jz_plan_free(plan)


def test_server_thermalises_a_large_state_from_hbm(ctx):
    """2D L = 96, L_t = 4L (73,728 sites: a Swendsen-Wang state beyond shared
    memory, a Metropolis lattice within it) through the server: spins and
    HBM slices charged to the job, the oracle's bits."""
    j = wl.Job(2, 96, 384, BC2, 30, 3, 1, 5, seed=23, n_therm=3, therm_update=H)
    server = jz.jz_server_create(ctx, 1 << 30, 2)
    try:
        i = jz.jz_submit(server, params(j))
        assert jz.jz_wait(server, i, 600.0).status == 0
        w = np.empty(j.n_traj, dtype=np.int64)
        jz.jz_server_work(server, i, w)
    finally:
        jz.jz_server_free(server)
    Wo, _ = oracle_run(j)
    np.testing.assert_array_equal(w, Wo)


def test_entry_points_that_do_not_serve_it_refuse(ctx):
    j = JOBS[0]
    p = params(j)
    w = torch.empty(j.n_traj, dtype=torch.int64, device="cuda")
    for call in (lambda: jz.jarzynski_run_plain(ctx, p, w),
                 lambda: jz.jarzynski_run_noalloc(p, w, None)):
        with pytest.raises(jz.IsingError) as e:
            call()
        assert e.value.code == jz.ISING_ERR_UNSUPPORTED
    bad = jz.make_params(2, 8, 8, BC2, 1, 2, 1, 2, 0, therm_update=2)
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_ex(ctx, bad, torch.empty(2, dtype=torch.int64, device="cuda"))
    assert e.value.code == jz.ISING_ERR_ARG
