"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host only).

A copy of jz_oracle.c instrumented with -fsanitize=address,undefined (errors
abort the process) runs small trajectories of every method option (the
Swendsen-Wang thermalisation before a Metropolis protocol included) in a child
process that preloads the ASan runtime; it must finish cleanly and give the
bits of the uninstrumented oracle."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

import oracle

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
lib = oracle.load_library(sys.argv[2])
cases = [dict(), dict(update=1), dict(protocol=2, d=3, L=4, L_t=4, l=1, n_step=8),
         dict(n_replica=3), dict(whole=True, update=1, l=4), dict(direction=-1),
         dict(L=6, L_t=4, l=5), dict(therm_update=1), dict(therm_update=1, d=3, L=4, L_t=4, l=1)]
out = []
for c in cases:
    kw = dict(d=2, L=8, L_t=8, beta=0.44068679350977147, l=3, n_step=6, n_sweep=1, n_traj=5, seed=9)
    kw.update(c)
    args = [kw.pop(k) for k in ("d", "L", "L_t", "beta", "l", "n_step", "n_sweep", "n_traj", "seed")]
    W, S = oracle.run(*args, n_therm=5, want_spins=True, lib=lib, **kw)
    out.append([W.tolist(), int(S.astype(np.int64).sum())])
print(json.dumps(out))
"""


def _gcc_runtime(name):
    try:
        path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True,
                              text=True, check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    asan = _gcc_runtime("libasan.so")
    if asan is None:
        pytest.skip("no ASan runtime for gcc on this host")
    lib = str(tmp_path / "liboracle_san.so")
    oracle.build(out=lib, sanitize=True)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, lib], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr
    got = json.loads(r.stdout.strip().splitlines()[-1])
    # the same cases through the uninstrumented oracle in this process
    r2 = subprocess.run([sys.executable, "-c", CHILD, ROOT, oracle.build()], capture_output=True,
                        text=True, env=dict(os.environ, OMP_NUM_THREADS="2"), timeout=600)
    assert r2.returncode == 0, r2.stderr[-2000:]
    assert got == json.loads(r2.stdout.strip().splitlines()[-1])
