"""Host-only services of the library (no GPU): the persisted autotune cache
and the server's per-job JSON line."""
import json
import math

import pytest

import paper_2304_03311_gb300 as jz
from paper_2304_03311_gb300 import build as jzbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    jzbuild.build()
    return jz.load()


def test_tune_cache_buckets_by_log2_trajectories():
    c = jz.TuneCache()
    c.put("NVIDIA GB300", 2, 64, 64, 2, 16384, 512)
    assert c.get("NVIDIA GB300", 2, 64, 64, 2, 16384) == 512
    assert c.get("NVIDIA GB300", 2, 64, 64, 2, 32767) == 512      # same power-of-two bucket
    assert c.get("NVIDIA GB300", 2, 64, 64, 2, 32768) is None     # next bucket
    assert c.get("NVIDIA GB300", 2, 64, 64, 0, 16384) == 512      # n_replica 0 means 2
    assert c.get("NVIDIA GB300", 2, 64, 64, 3, 16384) is None     # other replica count
    assert c.get("NVIDIA GB200", 2, 64, 64, 2, 16384) is None     # other GPU
    assert c.get("NVIDIA GB300", 3, 64, 64, 2, 16384) is None
    c.put("NVIDIA GB300", 2, 64, 64, 2, 20000, 384)               # same key: replaced
    assert c.get("NVIDIA GB300", 2, 64, 64, 2, 16384) == 384
    assert len(c) == 1


def test_tune_cache_file_round_trip(tmp_path):
    c = jz.TuneCache()
    entries = [("NVIDIA GB300", 2, 64, 64, 2, 16384, 512), ("NVIDIA GB300", 3, 16, 16, 2, 4096, 256),
               ("NVIDIA GB300", 2, 16, 16, 2, 1000, 32), ("Other GPU", 2, 32, 32, 3, 1024, 128),
               ("NVIDIA GB300", 2, 200, 200, 2, 4096, 0)]      # 0: the default shape won
    for e in entries:
        c.put(*e)
    path = tmp_path / "tune.json"
    c.save(path)
    doc = json.loads(path.read_text())             # the file is JSON
    assert doc["version"] == 1 and len(doc["entries"]) == 5
    assert {"gpu", "d", "L", "L_t", "n_replica", "traj_bucket", "cta_threads"} == set(doc["entries"][0])
    d = jz.TuneCache()
    d.load(path)
    assert len(d) == 5
    for gpu, dd, L, Lt, n, nt, t in entries:
        assert d.get(gpu, dd, L, Lt, n, nt) == t
    # loading merges, later files win
    e = jz.TuneCache()
    e.put("NVIDIA GB300", 2, 64, 64, 2, 16384, 64)
    e.put("NVIDIA GB300", 2, 8, 8, 2, 16, 32)
    e.load(path)
    assert len(e) == 6 and e.get("NVIDIA GB300", 2, 64, 64, 2, 16384) == 512
    with pytest.raises(jz.IsingError):
        e.put("NVIDIA GB300", 2, 64, 64, 2, 16384, -1)   # no negative CTA size


def test_tune_cache_rejects_bad_files(tmp_path):
    c = jz.TuneCache()
    with pytest.raises(jz.IsingError) as err:
        c.load(tmp_path / "missing.json")
    assert err.value.code == jz.ISING_ERR_NOT_FOUND
    bad = tmp_path / "bad.json"
    bad.write_text('{"version": 1, "entries": [\n{"gpu": "x", "d": 5}\n]}\n')
    with pytest.raises(jz.IsingError) as err:
        c.load(bad)
    assert err.value.code == jz.ISING_ERR_ARG
    truncated = tmp_path / "trunc.json"
    truncated.write_text('{"version": 1, "entries": [\n')
    with pytest.raises(jz.IsingError):
        c.load(truncated)
    assert len(c) == 0                               # nothing merged from a bad file


def test_result_json_line():
    p = jz.make_params(2, 64, 64, 0.44068679350977147, 7, 1000, 2, 256, seed=11,
                       therm_update=jz.SW_THERM)
    r = jz.JzResult(status=0, log_ratio=-0.0123, delta_S2=0.0123, delta_S2_err=0.0004,
                    submit_s=1.0, start_s=1.5, done_s=3.5, updates=10**12)
    line = jz.jz_result_json(42, p, r)
    doc = json.loads(line)
    assert doc["job"] == 42 and doc["L"] == 64 and doc["l"] == 7 and doc["n_traj"] == 256
    assert doc["seed"] == 11 and doc["n_replica"] == 2 and doc["status"] == 0
    assert doc["update"] == 0 and doc["therm_update"] == 1
    assert doc["delta_S2"] == 0.0123 and doc["delta_S2_err"] == 0.0004
    assert math.isclose(doc["latency_s"], 2.5) and doc["spin_updates"] == 10**12
    assert math.isclose(doc["spin_updates_per_s"], 10**12 / 2.0)
    # a failed job has no estimates
    r.status = jz.ISING_ERR_NOMEM
    doc = json.loads(jz.jz_result_json(43, p, r))
    assert doc["status"] == jz.ISING_ERR_NOMEM and doc["delta_S2"] is None
    assert doc["spin_updates_per_s"] is None
    import ctypes
    small = ctypes.create_string_buffer(16)
    assert jz.load().jz_result_json(1, ctypes.byref(p), ctypes.byref(r), small, 16) == jz.ISING_ERR_ARG
