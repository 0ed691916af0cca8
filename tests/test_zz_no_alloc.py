"""The allocation-free entry point jarzynski_run_noalloc.

It serves callers that may not allocate device memory (a plug-in whose host
application's allocator already holds the GPU's memory, or a loop that must not
stall in cudaMalloc / cudaFree).  Its scratch lives in one fixed 1 MiB device
array inside the library.  These tests call it through the C ABI twice in a row,
on different shapes and protocol lengths so that the second call runs over the
first call's leftovers (both updates, protocols short and long enough to need
several staging launches), and require the same W_int bits as the allocating
entry point jarzynski_run_ex.  The file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

import paper_2304_03311_gb300 as jz  # noqa: E402
from paper_2304_03311_gb300 import build as jzbuild  # noqa: E402
from paper_2304_03311_gb300 import workloads as wl  # noqa: E402

JOBS = [
    wl.Job(2, 16, 16, wl.BETA_C_2D, 4, 60, 1, 70, seed=3, n_therm=40),
    wl.Job(3, 8, 8, wl.BETA_C_3D, 2, 25, 2, 41, seed=4, n_therm=20, direction=-1),
    # Swendsen-Wang: two bond thresholds per step, one CTA per trajectory;
    # N = 4000 (8000 words) needs two staging launches of the scratch
    wl.Job(2, 8, 8, wl.BETA_C_2D, 3, 4000, 1, 9, seed=5, n_therm=6, update=1),
    # a protocol long enough for several staging launches (16000 words)
    wl.Job(2, 16, 16, wl.BETA_C_2D, 7, 1000, 1, 33, seed=6, n_therm=3),
]


def _params(job):
    return jz.make_params(job.d, job.L, job.L_t, job.beta, job.l, job.n_step, job.n_sweep,
                          job.n_traj, job.seed, n_therm=job.n_therm, direction=job.direction,
                          traj0=job.traj0, update=job.update)


def _reference(job):
    ctx = jz.ising_replica_init(0, 0, None)
    try:
        w = torch.empty(job.n_traj, dtype=torch.int64, device="cuda")
        jz.jarzynski_run_ex(ctx, _params(job), w, None)
        jz.ising_sync(ctx)
        return w.cpu().numpy()
    finally:
        jz.ising_replica_free(ctx)


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row():
    jzbuild.build()
    refs = [_reference(job) for job in JOBS]
    stream = torch.cuda.Stream()
    outs = [torch.full((job.n_traj,), -7, dtype=torch.int64, device="cuda") for job in JOBS]
    torch.cuda.synchronize()
    for job, out, ref in zip(JOBS, outs, refs):
        jz.jarzynski_run_noalloc(_params(job), out, stream.cuda_stream)
        stream.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
    # after the first call's set-up, further calls leave the device's free
    # memory as it was; the figure is device-wide, so a change made by another
    # process gets one retry
    again = torch.full((JOBS[0].n_traj,), -7, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    same = False
    for _ in range(2):
        free_before, _ = torch.cuda.mem_get_info()
        jz.jarzynski_run_noalloc(_params(JOBS[0]), again, stream.cuda_stream)
        stream.synchronize()
        free_after, _ = torch.cuda.mem_get_info()
        np.testing.assert_array_equal(again.cpu().numpy(), refs[0])
        if free_after == free_before:
            same = True
            break
    assert same


def test_noalloc_rejects_what_it_cannot_hold():
    jzbuild.build()
    out = torch.empty(8, dtype=torch.int64, device="cuda")
    too_long = jz.make_params(3, 8, 8, 0.2, 1, 10921, 1, 8, 0)      # 10921 * 24 words > 1 MiB
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_noalloc(too_long, out, None)
    assert e.value.code == jz.ISING_ERR_SCRATCH_LIMIT
    host_out = torch.empty(8, dtype=torch.int64)
    with pytest.raises(jz.IsingError) as e:
        jz.jarzynski_run_noalloc(jz.make_params(2, 8, 8, 0.4, 1, 5, 1, 8, 0), host_out, None)
    assert e.value.code == jz.ISING_ERR_ARG
