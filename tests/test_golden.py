"""Oracle against the stored fixtures under tests/golden/.

exact_delta.txt is a closed form (arXiv 2104.13347 Sec. II.A: gain 1/(4 pi d)
at an integer delay); the tiny_room files were written by
tests/golden/make_golden.py from the oracle alone and guard against drift.
"""
import ast
import os

import numpy as np

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    params, vals = None, []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            if line.startswith("# arXiv") and "params:" in line:
                params = ast.literal_eval(line.split("params:", 1)[1].strip())
            elif not line.startswith("#") and line.strip():
                vals.append(line.split())
    return params, vals


def test_exact_delta_fixture():
    _, vals = _read("exact_delta.txt")
    h = oracle.rir([5, 4, 3], [0.0] * 6, [2.0, 1.5, 1.5], [3.0, 1.5, 1.5], 16384.0, 256.0, 0,
                   81, oracle.FD_HANN_SINC, 256)
    ref = np.zeros(256)
    for idx, v in vals:
        ref[int(idx)] = float(v)
    np.testing.assert_array_equal(h, ref)
    assert float(vals[0][1]) == 1.0 / (4.0 * np.pi)


def test_oracle_regression_fixtures():
    for name in ("tiny_room_hann81.txt", "tiny_room_lagrange8.txt"):
        p, vals = _read(name)
        ref = np.array([float(v[0]) for v in vals])
        h = oracle.rir(p["dims"], p["beta"], p["src"], p["mic"], p["fs"], p["c"], p["order"],
                       p["n_taps"], p["fd_kind"], p["rir_len"])
        np.testing.assert_allclose(h, ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())
