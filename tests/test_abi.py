"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares.  No compute calls: these tests run without a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from conftest import ROOT

import paper_2304_03311_gb300 as jz
from paper_2304_03311_gb300 import build as jzbuild


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            if not m.group(0).lstrip().startswith(("#", "typedef", "return")):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    jzbuild.build()
    return jz.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ising_replica_init", "ising_replica_free", "jarzynski_run",
                     "jarzynski_run_ex", "jarzynski_run_batch", "estimator_reduce",
                     "ising_strerror", "ising_sync", "jz_params_default"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", jz.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_device_code_is_built_for_sm103a_only():
    # every translation unit and the link use exactly one -gencode, sm_103a
    assert jzbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_layout_matches_header(lib):
    # jz_params: 4 ints, double, 6 ints, long long, uint64, 4 ints -> 80 bytes
    assert ctypes.sizeof(jz.JzParams) == 80
    offs = {name: getattr(jz.JzParams, name).offset for name, _ in jz.JzParams._fields_}
    assert offs == {"d": 0, "L": 4, "L_t": 8, "update": 12, "beta": 16, "l": 24, "n_step": 28,
                    "n_sweep": 32, "n_therm": 36, "n_traj": 40, "direction": 44, "traj0": 48,
                    "seed": 56, "protocol": 64, "n_replica": 68, "whole": 72,
                    "therm_update": 76}
    p = jz.jz_params_default()
    assert (p.n_therm, p.n_sweep, p.direction, p.traj0, p.seed) == (1000, 1, 1, 0, 0)
    assert p.update == jz.METROPOLIS
    assert p.protocol == 1
    assert (p.n_replica, p.whole, p.therm_update) == (2, 0, 0)


def test_struct_layout_as_the_c_compiler_lays_it_out(tmp_path):
    """The ctypes mirror of jz_params against offsetof / sizeof from gcc on the
    header itself."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    names = [n for n, _ in jz.JzParams._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"isingjz.h\"\n"
                   "int main(void) {\n  printf(\"%zu\\n\", sizeof(jz_params));\n" +
                   "".join(f'  printf("%zu\\n", offsetof(jz_params, {n}));\n' for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(jz.JzParams)
    assert got[1:] == [getattr(jz.JzParams, n).offset for n in names]


def test_strerror_and_host_only_entry_points(lib):
    assert jz.ising_strerror(0) == "ok"
    assert "even" in jz.ising_strerror(jz.ISING_ERR_ODD_EXTENT)
    assert jz.ising_strerror(12345) == "unknown error"
    assert lib.jz_params_default(None) == jz.ISING_ERR_ARG
    assert lib.ising_replica_init(None, 0, 0, None) == jz.ISING_ERR_ARG
    lib.ising_replica_free(None)      # NULL is a no-op
    assert lib.ising_sync(None) == jz.ISING_ERR_ARG


def test_release_build_has_no_bounds_status(lib):
    import ctypes
    a, b = ctypes.c_uint(), ctypes.c_uint()
    assert lib.ising_bounds_status(ctypes.byref(a), ctypes.byref(b), 0) == jz.ISING_ERR_UNSUPPORTED
