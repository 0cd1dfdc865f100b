"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer
(host build, CPU only): every entry point on small and edge-case inputs
(lattice order 0, one-sample RIRs, 1- and 255-tap filters, the 2- and
8-tap Lagrange filters, the delay-limited order, OpenMP batches,
convolutions of one sample, frames reaching past either end of the signal)
runs without a memory or undefined-behaviour report and gives bit for bit
the results of the normal build."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, numpy as np, oracle
out = {}
def put(name, *arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    out[name] = h.hexdigest()
dims, beta = (4.3, 3.1, 2.7), [0.9, 0.7, 0.8, 0.95, 0.6, 0.85]
src, mic = (1.1, 2.2, 0.9), (3.0, 0.7, 1.8)
for order, L, taps, kind in [(0, 1, 81, 0), (2, 64, 81, 0), (2, 700, 1, 0), (1, 300, 255, 0),
                             (2, 500, 8, 1), (2, 500, 2, 1), (-1, 300, 81, 0)]:
    h, st = oracle.rir(dims, beta, src, mic, 16000.0, 343.0, order, taps, kind, L,
                       return_stats=True)
    put(f"rir_{order}_{L}_{taps}_{kind}", h, np.array(list(st.values())))
put("auto_order", np.array([oracle.auto_order(dims, src, mic, 16000.0, 343.0, 81, 900)]))
im = oracle.images(dims, beta, src, mic, 16000.0, 343.0, 2)
put("images", im["idx"], im["d"], im["tau"], im["f"], im["amp"], im["k0"])
rooms = [dict(dims=np.array(dims), beta=np.array(beta), src=np.array(src),
              mics=np.array([mic, (1.0, 1.0, 1.0), (2.0, 2.5, 0.4)]), fs=16000.0, c=343.0,
              order=o, n_taps=81, fd_kind=0, rir_len=L) for o, L in [(1, 200), (-1, 333)]]
hs, st = oracle.rir_batch(rooms, n_threads=2)
put("rir_batch", *hs, st)
for f in (0.0, 0.3, -0.5, 0.4999):
    put(f"hann_{f}", oracle.hann_sinc_taps(f, 81), oracle.hann_sinc_taps(f, 1))
for D in (3.0, 3.5, 3.999):
    put(f"lagrange_{D}", oracle.lagrange_taps(D, 8))
rng = np.random.default_rng(5)
s1, h1 = rng.standard_normal(1), rng.standard_normal(1)
s, h = rng.standard_normal(257), rng.standard_normal(33)
put("convolve", oracle.convolve(h1, s1), oracle.convolve(h, s),
    oracle.convolve_at(h, s, np.array([0, 5, 288])))
put("convolve_batch", *oracle.convolve_batch([h[None, :], np.stack([h, h[::-1]])], [s, s1],
                                             n_threads=2))
put("splitmix", np.array([oracle.splitmix64(1234567, i) for i in range(4)], np.uint64))
put("gauss", np.array([oracle.gauss(9, 3, 1, t) for t in range(7)]))
put("uniforms", *oracle.uniforms(9, 3, 1, 5, 11))
y = rng.standard_normal((3, 50))
put("add_noise", *oracle.add_noise(y.copy(), 12.0, 9, 4)[:1], *oracle.add_noise(y.copy(), 300.0, 9, 4)[:1])
for t0, n, snr in [(-60, 40, 10.0), (45, 20, float("nan")), (0, 1, 5.0), (-5, 70, float("inf"))]:
    put(f"frame_{t0}_{n}", oracle.frame(y, t0, n, snr, 9, 2)[0])
print(json.dumps(out))
"""


def run_script(tmp, sanitize):
    env = dict(os.environ, PYTHONPATH=ROOT, ORACLE_BUILD=str(tmp / ("san" if sanitize else "plain")),
               OMP_NUM_THREADS="2")
    env.pop("ORACLE_SRC", None)
    env.pop("ORACLE_SANITIZE", None)
    if sanitize:
        asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                              text=True).stdout.strip()
        if not os.path.isabs(asan) or not os.path.exists(asan):
            pytest.skip("no ASan runtime for gcc")
        env.update(ORACLE_SANITIZE="1", LD_PRELOAD=asan,
                   ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
                   UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    return subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True,
                          text=True, timeout=600)


def test_oracle_clean_under_asan_and_ubsan(tmp_path):
    plain = run_script(tmp_path, False)
    assert plain.returncode == 0, plain.stderr[-2000:]
    san = run_script(tmp_path, True)
    assert san.returncode == 0, san.stderr[-4000:]
    assert "runtime error" not in san.stderr and "AddressSanitizer" not in san.stderr
    assert os.path.exists(tmp_path / "san" / "libism_oracle_san.so")
    a, b = json.loads(plain.stdout), json.loads(san.stdout)
    assert len(a) > 25 and a == b
