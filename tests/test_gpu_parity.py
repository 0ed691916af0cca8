"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bit-exact: W_int per trajectory and the final spins, for identical parameters
and seed (the work and the spins are exact integers).  Estimator: within
|a - b| <= 1e-12 max(|a|, |b|) + 1e-14 (the absolute floor covers Delta S_2 ~ 0).
Small cases span several tiles and ragged rows (L/2 not a multiple of 4), both
directions, 2D and 3D, l = 0 and l = L-1, beta = 0, L_t = 2 and L = 2; the full
benchmark workloads are checked on trajectories sampled from the very launch
the benchmark times.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.estimator as oest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

import paper_2304_03311_gb300 as jz  # noqa: E402
from paper_2304_03311_gb300 import build as jzbuild  # noqa: E402
from paper_2304_03311_gb300 import workloads as wl  # noqa: E402

BC2, BC3 = wl.BETA_C_2D, wl.BETA_C_3D


def close(a, b):
    return abs(a - b) <= 1e-12 * max(abs(a), abs(b)) + 1e-14


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


def gpu_run(ctx, job, spins=True, on_device=True):
    V = job.sites
    dev = "cuda" if on_device else "cpu"
    w = torch.empty(job.n_traj, dtype=torch.int64, device=dev)
    s = torch.empty(job.n_traj * V, dtype=torch.int8, device=dev) if spins else None
    p = jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                       job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                       traj0=job.traj0)
    jz.jarzynski_run_ex(ctx, p, w, s)
    jz.ising_sync(ctx)
    return w.cpu().numpy(), (s.cpu().numpy().reshape(job.n_traj, -1) if spins else None)


def oracle_run(job, traj0=None, n_traj=None, spins=True):
    W, S = oracle.run(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                      n_traj if n_traj is not None else job.n_traj, job.seed,
                      n_therm=job.n_therm, direction=job.direction,
                      traj0=job.traj0 if traj0 is None else traj0, want_spins=spins)
    return W, (S.reshape(len(W), -1) if spins else None)


SMALL = [
    wl.Job(2, 16, 16, BC2, 4, 20, 1, 40, seed=0, n_therm=30),
    wl.Job(2, 12, 6, 0.5, 0, 7, 2, 33, seed=5, n_therm=5),              # L/2 = 6: ragged
    wl.Job(2, 10, 4, 0.3, 9, 5, 1, 17, seed=6, n_therm=4, direction=-1),  # l = L-1, reverse
    wl.Job(2, 2, 2, BC2, 1, 3, 1, 50, seed=7, n_therm=3),               # smallest lattice
    wl.Job(2, 4, 2, BC2, 2, 4, 3, 21, seed=8, n_therm=2, direction=-1),  # L_t = 2
    wl.Job(2, 64, 64, BC2, 30, 6, 2, 5, seed=0, n_therm=6),
    wl.Job(2, 34, 8, 0.45, 17, 5, 1, 6, seed=9, n_therm=3),             # L/2 = 17
    wl.Job(2, 256, 8, BC2, 100, 3, 1, 3, seed=10, n_therm=2),           # 32 words per row
    wl.Job(3, 4, 4, BC3, 1, 6, 1, 20, seed=11, n_therm=5),
    wl.Job(3, 6, 4, 0.25, 5, 4, 1, 9, seed=12, n_therm=3, direction=-1),  # 3D ragged
    wl.Job(3, 16, 8, 0.22165455, 7, 10, 1, 12, seed=13, n_therm=10),
    wl.Job(3, 2, 2, 0.3, 0, 3, 2, 40, seed=14, n_therm=2),
    wl.Job(2, 16, 16, 0.0, 4, 8, 1, 16, seed=15, n_therm=4),            # beta = 0
    wl.Job(2, 16, 16, 2.0, 4, 8, 1, 16, seed=16, n_therm=4),            # deep ordered phase
    wl.Job(2, 16, 8, BC2, 3, 9, 1, 12, seed=2**64 - 1, n_therm=3, traj0=123456),
]


@pytest.mark.parametrize("job", SMALL, ids=lambda j: f"d{j.d}L{j.L}Lt{j.L_t}l{j.l}dir{j.direction}")
def test_bit_exact_work_and_spins(ctx, job):
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def slice_words(job):
    """Spin words per time slice: 8 sites per word, L_y rows."""
    return ((job.L // 2 + 7) // 8) * (job.L if job.d == 3 else 1)


def params_of(job, **kw):
    return jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                          kw.get("n_traj", job.n_traj), job.seed, n_therm=job.n_therm,
                          direction=job.direction, traj0=job.traj0)


@pytest.mark.parametrize("job", [j for j in SMALL if slice_words(j) <= 32],
                         ids=lambda j: f"d{j.d}L{j.L}Lt{j.L_t}l{j.l}dir{j.direction}")
def test_bit_exact_in_warp_teams(job):
    """A few trajectories by default run one team per CTA, spread over more
    SMs; the same jobs in warp teams (a CTA of 128 threads) give the oracle's
    bits too."""
    c = jz.ising_replica_init(0, 0, None)
    try:
        jz.ising_set_threads(c, job.d, job.L, job.L_t, 128)
        shape = jz.ising_launch_shape(c, params_of(job))
        Wg, Sg = gpu_run(c, job)
    finally:
        jz.ising_replica_free(c)
    assert shape["cta_threads"] == 128 or not shape["warp"]
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def test_default_shape_follows_occupancy(ctx):
    """The default launch shape: the benchmark scans keep their warp teams
    (one warp per 2D L = 64 trajectory, one per two 3D 16^3 ones, the 2D L = 16
    single job's one-row team); a narrow slice of a large lattice (2D L = 200,
    13 words, a 41.6 KB lattice per warp team) runs one team per CTA, whose
    CTAs keep more warps resident; a handful of trajectories takes teams of
    several warps."""
    def shape(d, L, Lt, n):
        return jz.ising_launch_shape(ctx, jz.make_params(d, L, Lt, 0.4, 1, 10, 1, n, 0))
    s2 = shape(2, 64, 64, 16384)
    assert s2["warp"] and s2["team_threads"] == 32 and not s2["hbm"]
    s1 = shape(2, 16, 16, 1000)
    assert s1["warp"] and s1["team_threads"] == 32
    s3 = shape(3, 16, 16, 4096)
    assert s3["warp"] and s3["team_threads"] == 32
    big = shape(2, 200, 200, 4096)
    assert not big["warp"] and big["teams"] == 1 and big["team_threads"] >= 128
    few = shape(2, 64, 64, 4)
    assert not few["warp"] and few["team_threads"] >= 64
    hbm = shape(2, 256, 2048, 32)
    assert hbm["hbm"] and not hbm["warp"] and hbm["team_threads"] == 512
    sw = jz.ising_launch_shape(ctx, jz.make_params(2, 64, 64, 0.4, 1, 10, 1, 8, 0,
                                                   update=jz.SWENDSEN_WANG))
    assert sw["cta_threads"] == 256 and sw["teams"] == 1


def test_default_cta_team_of_a_wide_lattice_is_bit_exact(ctx):
    """2D L = 200, L_t = 200: one team per CTA by default; the oracle's bits."""
    job = wl.Job(2, 200, 200, BC2, 60, 2, 1, 3, seed=31, n_therm=2)
    assert not jz.ising_launch_shape(ctx, params_of(job, n_traj=4096))["warp"]
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def test_largest_3d_lattice_fits_and_matches(ctx):
    """3D L = L_t = 48 (221 KB of spins in shared memory), few sweeps."""
    job = wl.Job(3, 48, 48, BC3, 20, 2, 1, 2, seed=3, n_therm=1)
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


@pytest.mark.parametrize("job", [SMALL[0], SMALL[2], SMALL[6], SMALL[9], SMALL[4]],
                         ids=["2d", "2d_rev", "2d_ragged", "3d_ragged_rev", "Lt2"])
def test_plain_baseline_is_bit_exact(ctx, job):
    """The plain one-lattice-per-launch form gives the same bits as the fused
    kernel and the oracle."""
    w = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
    s = torch.empty(job.n_traj * job.sites, dtype=torch.int8, device="cuda")
    p = jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                       job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                       traj0=job.traj0)
    jz.jarzynski_run_plain(ctx, p, w, s)
    jz.ising_sync(ctx)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(w.cpu().numpy(), Wo)
    np.testing.assert_array_equal(s.cpu().numpy().reshape(job.n_traj, -1), So)


@pytest.mark.parametrize("job", [SMALL[0], SMALL[1], SMALL[8], SMALL[9]],
                         ids=["2d", "2d_ragged", "3d", "3d_ragged_rev"])
def test_cta_size_does_not_change_results(job):
    """Every admissible CTA size, and the autotuner's choice, give the same bits."""
    c = jz.ising_replica_init(0, 0, None)
    try:
        ref, _ = gpu_run(c, job, spins=False)
        # words per time slice: 8 sites per word, L_y rows
        col = ((job.L // 2 + 7) // 8) * (job.L if job.d == 3 else 1)
        if col <= 32:       # warp teams: any multiple of 32
            sizes, bad = [32, 64, 128, 256, 512], 48
        else:               # one team per CTA: col * TS, TS <= L_t
            sizes = [col * ts for ts in (1, 2, 4, 8, 16) if ts <= job.L_t and col * ts <= 512]
            bad = col * (job.L_t + 1)
        for t in sizes:
            jz.ising_set_threads(c, job.d, job.L, job.L_t, t)
            W, _ = gpu_run(c, job, spins=False)
            np.testing.assert_array_equal(W, ref)
        with pytest.raises(jz.IsingError):
            jz.ising_set_threads(c, job.d, job.L, job.L_t, bad)
        p = jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                           job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction)
        best = jz.ising_autotune(c, p)
        assert best in sizes or best in (0, 128)        # 0: the default shape
        W, _ = gpu_run(c, job, spins=False)
        np.testing.assert_array_equal(W, ref)
    finally:
        jz.ising_replica_free(c)


def test_last_launch_time_covers_the_kernel_only():
    """ising_last_launch_ms: an error before any run call and after a call
    rejected by its argument checks; after a run, a positive device time no
    longer than the call's wall time."""
    import time
    c = jz.ising_replica_init(0, 0, None)
    try:
        with pytest.raises(jz.IsingError):
            jz.ising_last_launch_ms(c)
        job = SMALL[0]
        gpu_run(c, job, spins=False)   # warm-up: module load, first allocations
        t0 = time.perf_counter()
        gpu_run(c, job, spins=False)
        wall_ms = (time.perf_counter() - t0) * 1e3
        ms = jz.ising_last_launch_ms(c)
        assert 0.0 < ms <= wall_ms
        bad = jz.make_params(2, 15, 16, BC2, 4, 10, 1, 8, 0)   # odd L
        w = torch.empty(8, dtype=torch.int64, device="cuda")
        with pytest.raises(jz.IsingError):
            jz.jarzynski_run_ex(c, bad, w)
        with pytest.raises(jz.IsingError):
            jz.ising_last_launch_ms(c)
    finally:
        jz.ising_replica_free(c)


def test_host_and_device_outputs_agree(ctx):
    job = SMALL[1]
    Wd, Sd = gpu_run(ctx, job, on_device=True)
    Wh, Sh = gpu_run(ctx, job, on_device=False)
    np.testing.assert_array_equal(Wd, Wh)
    np.testing.assert_array_equal(Sd, Sh)


def test_batch_equals_single_runs(ctx):
    """Jobs of two shapes and several l in one call: each result equals its
    own run, bit for bit."""
    jobs = [wl.Job(2, 16, 8, BC2, l, 6, 1, 11 + l, seed=4, n_therm=5) for l in range(0, 16, 3)]
    jobs += [wl.Job(3, 4, 4, BC3, l, 5, 1, 7, seed=4, n_therm=3) for l in range(4)]
    jobs += [wl.Job(2, 16, 8, BC2, 2, 6, 1, 9, seed=99, n_therm=5)]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    params = [jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj,
                             j.seed, n_therm=j.n_therm) for j in jobs]
    jz.jarzynski_run_batch(ctx, params, outs)
    jz.ising_sync(ctx)
    for j, o in zip(jobs, outs):
        W1, _ = gpu_run(ctx, j, spins=False)
        np.testing.assert_array_equal(o.cpu().numpy(), W1)
        Wo, _ = oracle_run(j, spins=False)
        np.testing.assert_array_equal(W1, Wo)


def test_simple_entry_point(ctx):
    w = torch.empty(9, dtype=torch.int64, device="cuda")
    jz.jarzynski_run(ctx, 2, 8, 8, BC2, 3, 4, 1, 9, 21, w)
    jz.ising_sync(ctx)
    Wo, _ = oracle.run(2, 8, 8, BC2, 3, 4, 1, 9, 21, n_therm=1000)
    np.testing.assert_array_equal(w.cpu().numpy(), Wo)


@pytest.mark.parametrize("n", [1, 7, 1000, 16384])
def test_estimator_matches_oracle(ctx, n):
    rng = np.random.default_rng(n)
    wi = rng.integers(-400, 400, size=n).astype(np.int64) * 2
    for beta, N, direction in ((BC2, 1000, 1), (0.3, 7, -1), (0.0, 5, 1), (4.0, 3, 1)):
        lr, ds, err = jz.estimator_reduce(ctx, torch.from_numpy(wi).cuda(), n, beta, N,
                                          direction, 32)
        ref_lr = oest.log_mean_exp_neg(oest.work_values(wi, beta, N))
        ref_ds, ref_err = oest.delta_s2_with_error(wi, beta, N, direction, 32)
        assert close(lr, ref_lr)
        assert close(ds, ref_ds)
        if n >= 2:
            assert abs(err - ref_err) <= 1e-10 * max(err, ref_err) + 1e-14
        # host input buffer gives the same
        lr2, ds2, err2 = jz.estimator_reduce(ctx, wi, n, beta, N, direction, 32)
        assert (lr2, ds2, err2) == (lr, ds, err)


def test_argument_errors(ctx):
    w = torch.empty(4, dtype=torch.int64, device="cuda")
    cases = [((2, 7, 8, 0.4, 1, 5, 1, 4, 0), jz.ISING_ERR_ODD_EXTENT),
             ((2, 8, 7, 0.4, 1, 5, 1, 4, 0), jz.ISING_ERR_ODD_EXTENT),
             ((2, 8, 8, 0.4, 8, 5, 1, 4, 0), jz.ISING_ERR_L_RANGE),
             ((2, 8, 8, 0.4, -1, 5, 1, 4, 0), jz.ISING_ERR_L_RANGE),
             ((4, 8, 8, 0.4, 1, 5, 1, 4, 0), jz.ISING_ERR_UNSUPPORTED),
             ((2, 8, 8, -0.1, 1, 5, 1, 4, 0), jz.ISING_ERR_ARG),
             ((2, 8, 8, 0.4, 1, 0, 1, 4, 0), jz.ISING_ERR_ARG),
             ((2, 8, 8, 0.4, 1, 5, 1, 0, 0), jz.ISING_ERR_ARG),
             # a 3D time slice of L_y ceil(L/16) = 1024 words exceeds 512 threads
             ((3, 128, 4, 0.2, 1, 5, 1, 4, 0), jz.ISING_ERR_UNSUPPORTED)]
    for args, code in cases:
        with pytest.raises(jz.IsingError) as e:
            jz.jarzynski_run(ctx, *args, w)
        assert e.value.code == code


def test_hbm_budget_is_enforced(ctx):
    c = jz.ising_replica_init(0, 1024, None)
    try:
        w = torch.empty(4096, dtype=torch.int64)
        with pytest.raises(jz.IsingError) as e:
            jz.jarzynski_run(c, 2, 16, 16, BC2, 4, 200, 1, 4096, 0, w)
        assert e.value.code == jz.ISING_ERR_NOMEM
    finally:
        jz.ising_replica_free(c)


# ---------------------------------------------------------------- full size --
def _run_workload(ctx, workload):
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in workload.jobs]
    params = [jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj,
                             j.seed, n_therm=j.n_therm, direction=j.direction, traj0=j.traj0)
              for j in workload.jobs]
    jz.jarzynski_run_batch(ctx, params, outs)
    jz.ising_sync(ctx)
    return [o.cpu().numpy() for o in outs]


def _check_sampled(workload, results, picks):
    for ji, ti in picks:
        job = workload.jobs[ji]
        Wo, _ = oracle_run(job, traj0=job.traj0 + ti, n_traj=1, spins=False)
        assert results[ji][ti] == Wo[0], (ji, ti)


def _check_properties(workload, results):
    for job, W in zip(workload.jobs, results):
        bound = 2 * 2 * job.L ** (job.d - 2) * job.n_step
        assert np.all(np.abs(W) <= bound)
        assert np.all(W % 2 == 0)
        assert len(np.unique(W)) > 1


def test_full_config1_sampled(ctx):
    w = wl.config1()
    res = _run_workload(ctx, w)
    _check_properties(w, res)
    _check_sampled(w, res, [(0, 0), (0, 1), (0, 517), (0, 999)])


def test_full_config2_sampled(ctx):
    """The 31-transformation scan at full size, one launch as the benchmark
    runs it: one trajectory of every l (the first and last trajectory at the
    two ends of the scan) against the oracle, and the estimator of every l."""
    w = wl.config2()
    res = _run_workload(ctx, w)
    _check_properties(w, res)
    picks = [(l, (l * 523) % 16384) for l in range(31)]
    picks[-1] = (30, 16383)
    _check_sampled(w, res, picks)
    for job, W in zip(w.jobs, res):
        _, ds, err = jz.estimator_reduce(ctx, torch.from_numpy(W).cuda(), job.n_traj,
                                         job.beta, job.n_step, 1, 32)
        ref, ref_err = oest.delta_s2_with_error(W, job.beta, job.n_step, 1, 32)
        assert close(ds, ref)
        assert abs(err - ref_err) <= 1e-10 * max(err, ref_err) + 1e-14


def test_full_config3_sampled(ctx):
    """The 3D slab scan at full size: one trajectory of every l against the oracle."""
    w = wl.config3()
    res = _run_workload(ctx, w)
    _check_properties(w, res)
    _check_sampled(w, res, [(i, (i * 1013) % 4096) for i in range(7)] + [(7, 4095)])


@pytest.mark.parametrize("l", [0, 30])
def test_full_shape_spins_match_oracle(ctx, l):
    """Final spins at the benchmark's full 2D shape and protocol (L = L_t = 64,
    N = 1000 x 2 sweeps, 1000 thermalisation sweeps) for two trajectories."""
    job = wl.config2().jobs[l].with_(n_traj=2, traj0=9000)
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


@pytest.mark.parametrize("job", [
    wl.Job(2, 64, 4096, BC2, 5, 2, 1, 6, seed=21, n_therm=3),           # 262 KB per lattice
    wl.Job(3, 12, 1280, BC3, 4, 2, 1, 4, seed=22, n_therm=2, direction=-1),
    # the paper's-style 2D L = 256, L_t = 8L (512 KB per lattice): 152 resident
    # lattices exceed the part of L2 they keep, so their spins stream from DRAM
    wl.Job(2, 256, 2048, BC2, 100, 2, 1, 3, seed=24, n_therm=2),
], ids=["2d_L64_T4096", "3d_L12_T1280", "2d_L256_T2048"])
def test_lattice_beyond_shared_memory_runs_from_hbm(ctx, job):
    """Replica lattices too large for one CTA's shared memory keep their spins
    in an HBM slice per CTA; the bits stay those of the oracle."""
    Wg, Sg = gpu_run(ctx, job)
    Wo, So = oracle_run(job)
    np.testing.assert_array_equal(Wg, Wo)
    np.testing.assert_array_equal(Sg, So)


def test_large_narrow_lattice_runs_as_cta_team(ctx):
    """The paper's 2D lattice L = 128, L_t = 8L: 131 KB per trajectory leaves
    room for one warp team per CTA, so it runs as one CTA team; every CTA
    size gives the oracle's bits."""
    job = wl.Job(2, 128, 1024, BC2, 40, 2, 1, 3, seed=23, n_therm=2)
    Wo, So = oracle_run(job)
    c = jz.ising_replica_init(0, 0, None)
    try:
        for t in (0, 64, 256, 512):
            jz.ising_set_threads(c, 2, 128, 1024, t)
            Wg, Sg = gpu_run(c, job)
            np.testing.assert_array_equal(Wg, Wo)
            np.testing.assert_array_equal(Sg, So)
    finally:
        jz.ising_replica_free(c)


def test_device_code_was_built_for_sm103a():
    jzbuild.build()
    assert jz.ising_binary_version(0) == 103
