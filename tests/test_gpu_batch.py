"""GPU tests of the persistent batched launch (uneven lattices in one launch,
captured in a CUDA graph) and of the batched estimator.

Each job's W_int must be bit-identical to running it alone with the
per-trajectory kernel (and, for a sample, to the oracle); the graph replays
are deterministic; the batched estimator equals estimator_reduce.
"""
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


def _params(j):
    return jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                          n_therm=j.n_therm, direction=j.direction, traj0=j.traj0)


def _uneven_jobs():
    """2D and 3D, regular and ragged rows, both directions, several l, uneven
    trajectory counts and protocol lengths, one seed."""
    out = []
    for i, (d, L, Lt) in enumerate([(2, 32, 32), (2, 48, 16), (2, 12, 8), (2, 64, 64),
                                    (3, 8, 8), (3, 12, 12), (3, 16, 16), (3, 6, 4)]):
        beta = wl.BETA_C_2D if d == 2 else wl.BETA_C_3D
        for k, l in enumerate(sorted({1, L // 4, L // 2 - 1, L - 1})):
            out.append(wl.Job(d, L, Lt, beta, l, 5 + 3 * k, 1 + (k % 2), 3 + 5 * k + i, seed=7,
                              n_therm=6 + i, direction=1 if (i + k) % 3 else -1,
                              traj0=(i << 20) + 11 * k))
    return out


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


def _single(ctx, j):
    w = torch.empty(j.n_traj, dtype=torch.int64, device="cuda")
    jz.jarzynski_run_ex(ctx, _params(j), w)
    jz.ising_sync(ctx)
    return w.cpu().numpy()


@pytest.mark.parametrize("cta", [256, 288, 512, 0])
def test_persistent_batch_equals_single_runs(ctx, cta):
    jobs = _uneven_jobs()
    outs = [torch.full((j.n_traj,), -9, dtype=torch.int64, device="cuda") for j in jobs]
    est = torch.zeros(3 * len(jobs), dtype=torch.float64, device="cuda")
    plan = jz.jz_plan_create(ctx, [_params(j) for j in jobs], outs, est, cta)
    try:
        threads, grid, n_items = jz.jz_plan_info(plan)
        assert threads in (256, 288, 384, 512) and grid >= 1 and n_items >= len(jobs)
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
        first = [o.cpu().numpy().copy() for o in outs]
        for j, W in zip(jobs, first):
            np.testing.assert_array_equal(W, _single(ctx, j))
        e = est.cpu().numpy().reshape(-1, 3)
        for j, W, (lr, ds, err) in zip(jobs, first, e):
            ref_ds, ref_err = oest.delta_s2_with_error(W, j.beta, j.n_step, j.direction, 32)
            assert abs(ds - ref_ds) <= 1e-12 * max(abs(ds), abs(ref_ds)) + 1e-14
            if j.n_traj >= 2:
                assert abs(err - ref_err) <= 1e-10 * max(err, ref_err) + 1e-14
        # replaying the graph reproduces every bit
        for o in outs:
            o.fill_(-9)
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
        for o, W in zip(outs, first):
            np.testing.assert_array_equal(o.cpu().numpy(), W)
    finally:
        jz.jz_plan_free(plan)


def test_persistent_batch_matches_oracle_sample(ctx):
    jobs = _uneven_jobs()
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    plan = jz.jz_plan_create(ctx, [_params(j) for j in jobs], outs, None, 288)
    try:
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    for j, o in list(zip(jobs, outs))[::5]:
        Wo, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                           n_therm=j.n_therm, direction=j.direction, traj0=j.traj0)
        np.testing.assert_array_equal(o.cpu().numpy(), Wo)


def test_plan_runs_a_wide_lattice_as_one_cta_team(ctx):
    """2D L = 200 (41.6 KB per lattice): a 384-thread CTA holds only five of its
    warp teams, so the plan runs it as one team of the whole CTA, beside small
    lattices in warp teams; every job keeps the oracle's bits."""
    jobs = [wl.Job(2, 200, 200, wl.BETA_C_2D, 50, 2, 1, 3, seed=7, n_therm=2, traj0=1 << 20),
            wl.Job(2, 32, 32, wl.BETA_C_2D, 9, 6, 1, 40, seed=7, n_therm=5),
            wl.Job(3, 8, 8, wl.BETA_C_3D, 3, 5, 1, 21, seed=7, n_therm=4, traj0=2 << 20)]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    plan = jz.jz_plan_create(ctx, [_params(j) for j in jobs], outs, None, 384)
    try:
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    for j, o in zip(jobs, outs):
        Wo, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                           n_therm=j.n_therm, direction=j.direction, traj0=j.traj0)
        np.testing.assert_array_equal(o.cpu().numpy(), Wo)


def test_plan_rejects_mixed_seeds_and_host_outputs(ctx):
    jobs = _uneven_jobs()[:3]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    ps = [_params(j) for j in jobs]
    ps[1].seed = 8
    with pytest.raises(jz.IsingError) as e:
        jz.jz_plan_create(ctx, ps, outs, None, 256)
    assert e.value.code == jz.ISING_ERR_ARG
    host = [torch.empty(j.n_traj, dtype=torch.int64) for j in jobs]
    with pytest.raises(jz.IsingError) as e:
        jz.jz_plan_create(ctx, [_params(j) for j in jobs], host, None, 256)
    assert e.value.code == jz.ISING_ERR_ARG


def test_reduced_config4_in_one_launch(ctx):
    """The uneven benchmark batch (all 214 jobs, 9 shapes) with 1/64 of the
    trajectories and short protocols: one launch, every job equal to its own run."""
    w = wl.config4()
    jobs = [j.with_(n_traj=max(2, j.n_traj // 64), n_step=j.n_step // 50, n_therm=20)
            for j in w.jobs]
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in jobs]
    plan = jz.jz_plan_create(ctx, [_params(j) for j in jobs], outs, None, 0)
    try:
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    for j, o in list(zip(jobs, outs))[::7]:
        np.testing.assert_array_equal(o.cpu().numpy(), _single(ctx, j))


def test_full_config4_plan_one_trajectory_per_shape(ctx):
    """The uneven benchmark batch at full size (214 jobs, 9 lattice shapes, one
    persistent CUDA-graph launch with the autotuned CTA size, as the benchmark
    runs it): for every shape, one trajectory of its shortest job against the
    oracle, and the batched estimator of every job against the oracle's."""
    w = wl.config4()
    outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in w.jobs]
    est = torch.zeros(3 * len(w.jobs), dtype=torch.float64, device="cuda")
    plan = jz.jz_plan_create(ctx, [_params(j) for j in w.jobs], outs, est, 0)
    try:
        jz.jz_plan_launch(plan)
        jz.ising_sync(ctx)
    finally:
        jz.jz_plan_free(plan)
    res = [o.cpu().numpy() for o in outs]
    shapes = {}
    for i, j in enumerate(w.jobs):
        key = (j.d, j.L)
        if key not in shapes or j.n_step < w.jobs[shapes[key]].n_step:
            shapes[key] = i
    assert len(shapes) == 9
    for (d, L), i in sorted(shapes.items()):
        j = w.jobs[i]
        ti = j.n_traj // 2
        Wo, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, 1, j.seed,
                           n_therm=j.n_therm, direction=j.direction, traj0=j.traj0 + ti)
        assert res[i][ti] == Wo[0], (d, L, j.l)
    e = est.cpu().numpy().reshape(-1, 3)
    for j, W, (lr, ds, err) in zip(w.jobs, res, e):
        ref_ds, ref_err = oest.delta_s2_with_error(W, j.beta, j.n_step, j.direction, 32)
        assert abs(ds - ref_ds) <= 1e-12 * max(abs(ds), abs(ref_ds)) + 1e-14
        assert abs(err - ref_err) <= 1e-10 * max(err, ref_err) + 1e-14
