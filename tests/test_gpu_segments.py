"""Checkpoint / resume (jarzynski_run_segment): splitting the protocol
[0, N) into segments that hand over the spins and W_int through device
buffers gives the bits of one uninterrupted run, for both updates, both
protocols, n > 2, whole cuts and lattices held in HBM.  The random counter is
a function of the global sweep index, so nothing else has to be stored.
"""
import numpy as np
import pytest

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


def params(job, **kw):
    return jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                          job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                          traj0=job.traj0, n_replica=job.n_replica, whole=job.whole, **kw)


CASES = [
    (wl.Job(2, 16, 16, BC2, 4, 12, 2, 20, seed=1, n_therm=6), {}),
    (wl.Job(3, 6, 4, 0.25, 5, 12, 1, 9, seed=2, n_therm=3, direction=-1), {}),
    (wl.Job(2, 16, 16, BC2, 4, 12, 1, 10, seed=3, n_therm=5), dict(update=1)),
    (wl.Job(3, 8, 8, BC3, 2, 16, 1, 6, seed=4, n_therm=3), dict(update=1, protocol=2)),
    (wl.Job(3, 4, 4, BC3, 1, 12, 1, 12, seed=5, n_therm=3), dict(protocol=2)),
    (wl.Job(2, 8, 8, BC2, 3, 9, 1, 12, seed=6, n_therm=3, n_replica=3), {}),
    (wl.Job(2, 8, 8, BC2, 5, 9, 1, 12, seed=7, n_therm=3, whole=True), dict(update=1)),
    (wl.Job(2, 64, 4096, BC2, 5, 6, 1, 3, seed=8, n_therm=2), {}),            # HBM lattice
]


@pytest.mark.parametrize("job,opt", CASES, ids=[f"case{i}" for i in range(len(CASES))])
def test_segments_reproduce_one_run(ctx, job, opt):
    p = params(job, **opt)
    V = job.sites
    w_ref = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
    s_ref = torch.empty(job.n_traj * V, dtype=torch.int8, device="cuda")
    jz.jarzynski_run_ex(ctx, p, w_ref, s_ref)
    jz.ising_sync(ctx)
    w = torch.zeros(job.n_traj, dtype=torch.int64, device="cuda")
    s = torch.zeros(job.n_traj * V, dtype=torch.int8, device="cuda")
    cuts = [0, job.n_step // 3, job.n_step // 3 + 1, job.n_step]
    for a, b in zip(cuts[:-1], cuts[1:]):
        jz.jarzynski_run_segment(ctx, p, a, b, w, s)
        jz.ising_sync(ctx)
    assert torch.equal(w, w_ref)
    assert torch.equal(s, s_ref)


def test_segment_arguments(ctx):
    job = CASES[0][0]
    p = params(job)
    w = torch.zeros(job.n_traj, dtype=torch.int64, device="cuda")
    s = torch.zeros(job.n_traj * job.sites, dtype=torch.int8, device="cuda")
    for a, b in [(0, 0), (3, 2), (-1, 2), (0, job.n_step + 1)]:
        with pytest.raises(jz.IsingError) as e:
            jz.jarzynski_run_segment(ctx, p, a, b, w, s)
        assert e.value.code == jz.ISING_ERR_ARG
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_segment(ctx, p, 0, 2, w.cpu(), s)
    assert e.value.code == jz.ISING_ERR_ARG
