"""CPU oracle for the Jarzynski replica-gluing method (arXiv:2304.03311).

TEST INFRASTRUCTURE ONLY.  The oracle is the checker for the CUDA library, not a
part of it: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg of ``bench.py`` (and its ``--impl reference`` arm) may import or run it.  It
shares no code with ``paper_2304_03311_gb300``: the Monte Carlo trajectory is
plain C (``jz_oracle.c``), the exact solvers (``exact.py``) and the estimator
(``estimator.py``) are plain numpy, each function citing the passage it follows.

Pins (tests/test_oracle_*.py): Philox against Triton's CPU interpreter; exact
enumeration against Kaufman's finite-torus formula; the replica transfer matrix
against enumeration; the Monte Carlo work distribution against the exact path
measure; the estimator against high-precision arithmetic and closed forms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jz_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, out: str | None = None, mutant: int = 0,
          sanitize: bool = False) -> str:
    """Compile jz_oracle.c into oracle/liboracle.so with gcc (-O2, OpenMP).

    -ffp-contract=off keeps the threshold formula free of fused multiply-adds
    on every host, so the tables are the plain libm evaluation of the formula.
    ``mutant`` > 0 builds, at ``out``, a copy with one planted mistake (tests
    only, to show that the pins catch it).  ``sanitize`` builds, at ``out``, a
    copy instrumented with AddressSanitizer and UndefinedBehaviorSanitizer
    (errors abort; a process loading it must preload the ASan runtime).
    """
    path = out or _LIB_PATH
    if (mutant == 0 and not sanitize and not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    san = (["-fsanitize=address,undefined", "-fno-sanitize-recover=all",
            "-fno-omit-frame-pointer", "-g"] if sanitize else [])
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", f"-DORACLE_MUTANT={int(mutant)}"] + san + [
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def load_library(path: str):
    """ctypes handle on a built oracle library, signatures declared."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            _declare(lib)
            _lib = lib
    return _lib


def _declare(lib):
    """Declare the C signatures on a ctypes handle."""
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_run.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, ctypes.c_uint64, ctypes.c_longlong, ctypes.c_int,
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_philox4x32_10.argtypes = [ctypes.c_void_p] * 3
    lib.oracle_threshold_bulk.restype = ctypes.c_uint32
    lib.oracle_threshold_bulk.argtypes = [ctypes.c_double, ctypes.c_int]
    lib.oracle_threshold_cut.restype = ctypes.c_uint32
    lib.oracle_threshold_cut.argtypes = [ctypes.c_double, ctypes.c_longlong,
                                         ctypes.c_int]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle_run_update.restype = ctypes.c_int
    lib.oracle_run_update.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_longlong, ctypes.c_int,
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_run_full.restype = ctypes.c_int
    lib.oracle_run_full.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_longlong,
        ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_run_general.restype = ctypes.c_int
    lib.oracle_run_general.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_uint64, ctypes.c_longlong,
        ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_run_therm.restype = ctypes.c_int
    lib.oracle_run_therm.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_uint64, ctypes.c_longlong,
        ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_bond_threshold.restype = ctypes.c_uint32
    lib.oracle_bond_threshold.argtypes = [ctypes.c_double]


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11) for one counter and key."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def threshold_bulk(beta: float, m: int) -> int:
    return int(_load().oracle_threshold_bulk(beta, m))


def threshold_cut(beta: float, m: int, n_step: int) -> int:
    return int(_load().oracle_threshold_cut(beta, m, n_step))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def bond_threshold(x: float) -> int:
    """Swendsen-Wang bond threshold floor(2^32 (1 - e^-x)), x = 2K."""
    return int(_load().oracle_bond_threshold(x))


def run(d, L, L_t, beta, l, n_step, n_sweep, n_traj, seed, *, n_therm=1000,
        direction=1, traj0=0, n_threads=0, want_spins=False, lib=None, update=0,
        protocol=1, n_replica=2, whole=False, therm_update=None):
    """Run trajectories traj0..traj0+n_traj-1 of the transformation l -> l+1
    (direction=+1) or l+1 -> l (direction=-1); update 0 = checkerboard
    Metropolis, 1 = Swendsen-Wang clusters; protocol 1 switches every column
    of the cut together, protocol 2 one column y at a time (Appendix B; n_step
    a multiple of L_y).  n_replica replicas; whole=True runs Alba et al.'s
    whole-cut transformation (columns x < l switch from decoupled to glued,
    1 <= l <= L) instead of moving the end of region A by one column.
    therm_update (default: `update`) is the update of the n_therm
    thermalisation sweeps; Appendix A needs only an equilibrium start.

    Returns (W_int int64[n_traj], spins int8[n_traj, n_replica, L_t, L_y, L] or None).
    Follows section 3 (replica geometry and linear protocol) and Appendix A
    (work per step, update at lambda_{k+1}) of the paper.
    """
    lib = lib or _load()
    work = np.zeros(n_traj, dtype=np.int64)
    L_y = L if d == 3 else 1
    spins = (np.zeros((n_traj, n_replica, L_t, L_y, L), dtype=np.int8) if want_spins
             else None)
    th = int(update) if therm_update is None else int(therm_update)
    rc = lib.oracle_run_therm(int(d), int(L), int(L_t), float(beta), int(l), int(n_step),
                              int(n_sweep), int(n_therm), int(direction), int(update), th,
                              int(protocol), int(n_replica), int(bool(whole)),
                              int(seed) & 0xFFFFFFFFFFFFFFFF, int(traj0),
                              int(n_traj), int(n_threads), work.ctypes.data,
                              spins.ctypes.data if spins is not None else None)
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    return work, spins
