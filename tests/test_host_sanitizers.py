"""The library's host-only records (csrc/jz_records.cpp: the persisted autotune
cache and the per-job JSON line) under AddressSanitizer and
UndefinedBehaviorSanitizer, errors fatal.

A driver built with the file exercises every entry point with valid input
and with hostile input: malformed, truncated, empty and oversized cache
files, lines longer than the reader's buffer, GPU names with quotes,
backslashes, control bytes and more characters than a cache line holds,
NULL arguments, JSON buffers of every size from 0 up to the line's length,
and non-finite numbers.  It must exit cleanly, and its checks of the results
must hold."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include "isingjz.h"

static int fails = 0;
#define CHECK(c) do { if (!(c)) { std::printf("check failed: %s (line %d)\n", #c, __LINE__); ++fails; } } while (0)

static void write(const char* path, const std::string& text)
{
    FILE* f = std::fopen(path, "w");
    std::fwrite(text.data(), 1, text.size(), f);
    std::fclose(f);
}

int main(int argc, char** argv)
{
    const std::string dir = argv[1];
    const std::string good = dir + "/good.json", bad = dir + "/bad.json";
    jz_tune_cache* c = nullptr;
    CHECK(jz_tune_cache_create(&c) == ISING_OK);
    CHECK(jz_tune_cache_create(nullptr) == ISING_ERR_ARG);
    // names: ordinary, hostile bytes, and longer than a cache line holds
    std::string longname(5000, 'G');
    const char* names[] = {"NVIDIA GB300", "a\"b\\c\n\x01\x7f\xff", longname.c_str(), ""};
    for (int i = 0; i < 4; ++i)
        for (int d = 2; d <= 3; ++d)
            CHECK(jz_tune_cache_put(c, names[i], d, 8 * (i + 1), 16, 2, 1 << (i + 8), 32 * i) ==
                  ISING_OK);
    CHECK(jz_tune_cache_put(c, nullptr, 2, 8, 8, 2, 4, 32) == ISING_ERR_ARG);
    CHECK(jz_tune_cache_put(c, "x", 4, 8, 8, 2, 4, 32) == ISING_ERR_ARG);
    CHECK(jz_tune_cache_put(c, "x", 2, 8, 8, 2, 0, 32) == ISING_ERR_ARG);
    CHECK(jz_tune_cache_put(c, "x", 2, 8, 8, 2, 4, -1) == ISING_ERR_ARG);
    int n = 0, t = -5;
    CHECK(jz_tune_cache_size(c, &n) == ISING_OK && n == 8);
    CHECK(jz_tune_cache_get(c, longname.c_str(), 3, 24, 16, 2, 1 << 10, &t) == ISING_OK && t == 64);
    CHECK(jz_tune_cache_get(c, "nope", 2, 8, 16, 2, 256, &t) == ISING_ERR_NOT_FOUND);
    CHECK(jz_tune_cache_get(c, "x", 2, 8, 16, 2, 0, &t) == ISING_ERR_ARG);
    CHECK(jz_tune_cache_save(c, good.c_str()) == ISING_OK);
    CHECK(jz_tune_cache_save(c, (dir + "/no/such/dir.json").c_str()) == ISING_ERR_NOT_FOUND);
    jz_tune_cache* r = nullptr;
    CHECK(jz_tune_cache_create(&r) == ISING_OK);
    CHECK(jz_tune_cache_load(r, good.c_str()) == ISING_OK);   // what it wrote, it reads back
    CHECK(jz_tune_cache_size(r, &n) == ISING_OK && n == 8);
    CHECK(jz_tune_cache_get(r, longname.c_str(), 2, 24, 16, 2, 1 << 10, &t) == ISING_OK && t == 64);
    CHECK(jz_tune_cache_load(r, (dir + "/missing.json").c_str()) == ISING_ERR_NOT_FOUND);
    const std::string head = "{\"version\": 1, \"entries\": [\n";
    const std::string line = "{\"gpu\": \"g\", \"d\": 2, \"L\": 8, \"L_t\": 8, \"n_replica\": 2, "
                             "\"traj_bucket\": 3, \"cta_threads\": 64}\n";
    const std::string hostile[] = {
        "", "]}\n", head, head + line, head + line.substr(0, 40) + "\n]}\n",
        head + std::string(5000, 'x') + "\n]}\n",
        head + "{\"gpu\": \"" + std::string(3000, 'g') + "\", \"d\": 2}\n]}\n",
        head + "{\"gpu\": \"g\", \"d\": 2, \"L\": 99999999999999999999, \"L_t\": 8, "
               "\"n_replica\": 2, \"traj_bucket\": 3, \"cta_threads\": 64}\n]}\n",
        head + "{\"gpu\": \"g\", \"d\": 2, \"L\": 8, \"L_t\": 8, \"n_replica\": 2, "
               "\"traj_bucket\": 99, \"cta_threads\": 64}\n]}\n",
        head + line + "]}\n" + line, std::string("\0\0\0", 3), "{\"version\": 2}\n"};
    for (const std::string& h : hostile) {
        write(bad.c_str(), h);
        CHECK(jz_tune_cache_load(r, bad.c_str()) == ISING_ERR_ARG);
    }
    CHECK(jz_tune_cache_size(r, &n) == ISING_OK && n == 8);   // nothing merged from bad files
    write(bad.c_str(), head + line + "]}\n");
    CHECK(jz_tune_cache_load(r, bad.c_str()) == ISING_OK);
    CHECK(jz_tune_cache_get(r, "g", 2, 8, 8, 2, 8, &t) == ISING_OK && t == 64);
    jz_tune_cache_free(r);
    jz_tune_cache_free(c);
    jz_tune_cache_free(nullptr);

    // JSON line: every buffer size, and non-finite numbers
    jz_params p;
    CHECK(jz_params_default(&p) == ISING_OK);
    p.d = 2; p.L = 64; p.L_t = 64; p.beta = 0.44; p.l = 7; p.n_step = 1000; p.n_traj = 256;
    jz_result res;
    std::memset(&res, 0, sizeof res);
    res.status = ISING_OK; res.log_ratio = -0.01; res.delta_S2 = 0.01; res.delta_S2_err = 1e-4;
    res.submit_s = 1.0; res.start_s = 1.5; res.done_s = 3.0; res.updates = 1000000;
    char big[2048];
    const int len = jz_result_json(7, &p, &res, big, sizeof big);
    CHECK(len > 100 && (size_t)len == std::strlen(big));
    for (size_t m = 0; m <= (size_t)len + 1; ++m) {
        char* b = m ? new char[m] : nullptr;
        const int got = jz_result_json(7, &p, &res, b, m);
        CHECK(m > (size_t)len ? got == len : got == ISING_ERR_ARG);
        delete[] b;
    }
    p.beta = NAN;
    res.status = ISING_ERR_CUDA; res.log_ratio = INFINITY;
    CHECK(jz_result_json(8, &p, &res, big, sizeof big) > 0);
    CHECK(std::strstr(big, "nan") == nullptr && std::strstr(big, "inf") == nullptr);
    CHECK(jz_result_json(8, nullptr, &res, big, sizeof big) == ISING_ERR_ARG);
    CHECK(jz_result_json(8, &p, nullptr, big, sizeof big) == ISING_ERR_ARG);
    std::printf("fails %d\n", fails);
    return fails ? 1 : 0;
}
"""


def _compiler():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    return gxx


def test_records_under_asan_and_ubsan(tmp_path):
    gxx = _compiler()
    src = tmp_path / "driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "driver"
    csrc = os.path.join(ROOT, "paper_2304_03311_gb300", "csrc")
    # jz_params_default comes from the CUDA file; the driver gets its own copy
    # of that one function so that nothing links the CUDA runtime
    stub = tmp_path / "defaults.cpp"
    stub.write_text('#include <cstring>\n#include "isingjz.h"\n'
                    'extern "C" int jz_params_default(jz_params* p) {\n'
                    '  if (!p) return ISING_ERR_ARG;\n  std::memset(p, 0, sizeof *p);\n'
                    '  p->n_therm = 1000; p->n_sweep = 1; p->direction = 1; p->protocol = 1;\n'
                    '  p->n_replica = 2;\n  return ISING_OK;\n}\n')
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fno-omit-frame-pointer",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-I", os.path.join(ROOT, "include"), str(src), str(stub),
           os.path.join(csrc, "jz_records.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(exe), str(tmp_path)], capture_output=True, text=True, env=env,
                       timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails 0" in r.stdout
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr
