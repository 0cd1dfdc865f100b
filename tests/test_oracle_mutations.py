"""The oracle pins reject plausible mistakes.

Each case plants one slip in a scratch copy of the oracle's C source (a
swapped wall exponent, a sign flip in the delay split, a wrong lattice
spacing, a dropped distance term, a missing 4 pi, floor instead of
round-to-nearest, an off-by-one convolution index), builds it into a scratch
folder, and runs the pin suite against it in a subprocess: the suite must
fail.  Nothing here touches the real oracle build.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ism_oracle.c")

MUTATIONS = {
    "wall_exponent": ("pow(beta0, (double)abs(q - p))", "pow(beta0, (double)abs(q))"),
    "delay_sign": ("im.f = im.tau - k;", "im.f = k - im.tau;"),
    "lattice_spacing": ("(double)(2 * q) * L", "(double)(q) * L"),
    "dropped_term": ("double d2 = dx * dx + dy * dy;", "double d2 = dx * dx + dy * dx;"),
    "spreading": ("g / (4.0 * ORACLE_PI * im.d)", "g / (ORACLE_PI * im.d)"),
    "split_floor": ("double k = rint(im.tau);", "double k = floor(im.tau);"),
    "window_width": ("cos(ORACLE_PI * t / (double)(H + 1))", "cos(ORACLE_PI * t / (double)H)"),
    "conv_index": ("acc += h[k] * s[t - k];\n        y[t] = acc;",
                   "acc += h[k] * s[t - k + (k > 0)];\n        y[t] = acc;"),
    "noise_branch": ("return (t & 1) ? r * sin(2.0 * ORACLE_PI * u2) : r * cos(2.0 * ORACLE_PI * u2);",
                     "return r * cos(2.0 * ORACLE_PI * u2);"),
    "frame_padding": ("(t >= 0 && t < y_len) ? y[(int64_t)m * y_len + t] : 0.0;",
                      "(t >= 0 && t <= y_len) ? y[(int64_t)m * y_len + t] : 0.0;"),
    "auto_order": ("const double d_reach = ((double)rir_len + (double)n_taps) * c / fs;",
                   "const double d_reach = ((double)rir_len) * c / fs / 2.0;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_reject_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert old in text, f"mutation anchor for {name} not found"
    mut = tmp_path / "ism_oracle.c"
    mut.write_text(text.replace(old, new, 1))
    env = dict(os.environ, ORACLE_SRC=str(mut), ORACLE_BUILD=str(tmp_path / "build"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins accepted mutation {name}:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout
