"""The bounds-checked debug build (libisingjz_debug.so, -DJZ_BOUNDS_CHECK).

Every lattice word of the trajectory kernels and every cluster label and spin
bit of the Swendsen-Wang kernel is read and written through a check that
records an index outside its array in a device status word and skips the
access.  A clean run must leave the word at zero and give the release
library's (the oracle's) bits.  The binding binds one library per process, so
the debug run happens in a child process."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

from conftest import ROOT  # noqa: E402

CHILD = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2304_03311_gb300 import build as jzbuild
import paper_2304_03311_gb300 as jz
from paper_2304_03311_gb300 import workloads as wl
jzbuild.build(debug=True)
jz.use_debug_library()
jz.ising_bounds_status(clear=True)
BC2, BC3 = wl.BETA_C_2D, wl.BETA_C_3D
jobs = [
    (wl.Job(2, 16, 16, BC2, 4, 12, 1, 40, seed=0, n_therm=10), {}),
    (wl.Job(2, 12, 6, 0.5, 0, 7, 2, 33, seed=5, n_therm=5), {}),            # ragged rows
    (wl.Job(2, 10, 4, 0.3, 9, 5, 1, 17, seed=6, n_therm=4, direction=-1), {}),
    (wl.Job(2, 64, 64, BC2, 30, 4, 2, 5, seed=1, n_therm=4), {}),
    (wl.Job(3, 6, 4, 0.25, 5, 4, 1, 9, seed=12, n_therm=3, direction=-1), {}),
    (wl.Job(3, 16, 8, BC3, 7, 16, 1, 6, seed=13, n_therm=4), dict(protocol=2)),
    (wl.Job(2, 8, 8, BC2, 3, 6, 1, 16, seed=3, n_therm=4), dict(n_replica=3)),
    (wl.Job(2, 64, 4096, BC2, 5, 2, 1, 3, seed=21, n_therm=2), {}),          # lattice in HBM
    (wl.Job(2, 16, 16, BC2, 4, 10, 1, 8, seed=1, n_therm=6), dict(update=1)),
    (wl.Job(3, 4, 4, BC3, 1, 8, 1, 8, seed=2, n_therm=4), dict(update=1, protocol=2)),
    (wl.Job(2, 8, 8, BC2, 4, 6, 1, 8, seed=4, n_therm=4), dict(whole=True, update=1)),
]
ctx = jz.ising_replica_init(0, 0, None)
bad = []
for j, opt in jobs:
    w = torch.empty(j.n_traj, dtype=torch.int64, device="cuda")
    sites = opt.get("n_replica", 2) * j.L_t * j.L ** (j.d - 1)
    s = torch.empty(j.n_traj * sites, dtype=torch.int8, device="cuda")
    p = jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                       n_therm=j.n_therm, direction=j.direction, **opt)
    jz.jarzynski_run_ex(ctx, p, w, s)
    jz.ising_sync(ctx)
    W, S = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed,
                      n_therm=j.n_therm, direction=j.direction, want_spins=True, **opt)
    if not (np.array_equal(w.cpu().numpy(), W) and np.array_equal(s.cpu().numpy(), S.reshape(-1))):
        bad.append(str((j, opt)))
# a persistent plan of two shapes (the batch kernel's checks)
pj = [wl.Job(2, 32, 32, BC2, 5, 6, 1, 20, seed=7, n_therm=5), wl.Job(3, 8, 8, BC3, 2, 6, 1, 12, seed=7, n_therm=5)]
outs = [torch.empty(j.n_traj, dtype=torch.int64, device="cuda") for j in pj]
plan = jz.jz_plan_create(ctx, [jz.make_params(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep,
                                               j.n_traj, j.seed, n_therm=j.n_therm) for j in pj],
                         outs, None, 256)
jz.jz_plan_launch(plan)
jz.ising_sync(ctx)
jz.jz_plan_free(plan)
for j, o in zip(pj, outs):
    W, _ = oracle.run(j.d, j.L, j.L_t, j.beta, j.l, j.n_step, j.n_sweep, j.n_traj, j.seed, n_therm=j.n_therm)
    if not np.array_equal(o.cpu().numpy(), W):
        bad.append(str(j))
jz.ising_replica_free(ctx)
sites, index = jz.ising_bounds_status()
print(json.dumps({"lib": jz.lib_path(), "sites": sites, "index": index, "mismatch": bad}))
'''


def test_bounds_checked_build_runs_clean_and_bit_exact():
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["lib"].endswith("libisingjz_debug.so")
    assert out["mismatch"] == []
    assert out["sites"] == 0, out
