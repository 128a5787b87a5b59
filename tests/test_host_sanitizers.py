"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer: the CPU
oracle, and the library's host-only C++ (the sparse symbolic analysis and
the tuning cache).  Each is compiled with its driver under tests/sanitize/
and run; any sanitizer report aborts the run with a non-zero status."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
CSRC = os.path.join(ROOT, "paper_cs_0408029_gb300", "csrc")


def _build_and_run(cmd, exe):
    r = subprocess.run(cmd + ["-o", exe], capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("compiler without sanitizer runtimes: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stderr[-4000:]
    assert "runtime error" not in run.stderr and "Sanitizer" not in run.stderr, run.stderr[-4000:]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")
def test_oracle_under_sanitizers(tmp_path):
    _build_and_run(["gcc", "-std=c11", "-ffp-contract=off"] + SAN
                   + [os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c"), "-lm"],
                   str(tmp_path / "oracle_driver"))


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not found")
def test_library_host_code_under_sanitizers(tmp_path):
    _build_and_run(["g++", "-std=c++17"] + SAN
                   + ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC,
                      os.path.join(ROOT, "tests", "sanitize", "host_driver.cpp"),
                      os.path.join(CSRC, "sparse_sym.cpp"), os.path.join(CSRC, "tune_cache.cpp")],
                   str(tmp_path / "host_driver"))
