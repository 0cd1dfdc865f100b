"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer
(CPU only, no GPU): the host-side ABI tests -- argument checks, batch sizes,
the tuning-cache reader, the serving layer's admission limits and its
failure on an unusable device -- run against libism_san.so
(`python -m paper_2104_13347_gb300.build --host-sanitize`, host code
instrumented, device code unchanged) with the ASan runtime preloaded, and
pass without a memory or undefined-behaviour report."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_abi_suite_clean_under_asan_and_ubsan():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not found")
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                          text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime for gcc")
    from paper_2104_13347_gb300 import build
    lib = build.build(host_sanitize=True)
    env = dict(os.environ, PYTHONPATH=ROOT, ISM_LIB=os.path.basename(lib), LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_abi.py"),
                        "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "runtime error" not in out and "AddressSanitizer" not in out
    assert " passed" in r.stdout
    # the instrumented file is the one the binding mapped
    probe = ("from paper_2104_13347_gb300 import _lib\n_lib.load()\n"
             "print(any(l.rstrip().endswith('libism_san.so') for l in open('/proc/self/maps')))")
    p = subprocess.run([sys.executable, "-c", probe], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == "True", p.stdout + p.stderr[-2000:]
