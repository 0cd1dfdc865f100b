"""Writes the oracle regression fixtures in this folder.

Calls only the FP64 oracle (oracle/), never the CUDA path.  Run from the
repository root:  python tests/golden/make_golden.py
The fixtures freeze the oracle's output for two tiny rooms so that a later
change to the oracle's arithmetic shows up as a diff; any such change must
name, in its commit message, the passage of arXiv 2104.13347 (Sec. II.A) or
the reading of it that justifies it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402

CASES = {
    "tiny_room_hann81": dict(dims=[3.1, 2.3, 1.7], beta=[0.9, 0.8, 0.7, 0.6, 0.5, 0.4],
                             src=[0.7, 1.9, 0.4], mic=[2.2, 0.6, 1.3], fs=16000.0, c=343.0,
                             order=2, n_taps=81, fd_kind=oracle.FD_HANN_SINC, rir_len=256),
    "tiny_room_lagrange8": dict(dims=[3.1, 2.3, 1.7], beta=[0.9, 0.8, 0.7, 0.6, 0.5, 0.4],
                                src=[0.7, 1.9, 0.4], mic=[2.2, 0.6, 1.3], fs=16000.0, c=343.0,
                                order=2, n_taps=8, fd_kind=oracle.FD_LAGRANGE, rir_len=256),
}


def main():
    for name, p in CASES.items():
        h, st = oracle.rir(p["dims"], p["beta"], p["src"], p["mic"], p["fs"], p["c"],
                           p["order"], p["n_taps"], p["fd_kind"], p["rir_len"], return_stats=True)
        path = os.path.join(HERE, name + ".txt")
        with open(path, "w") as f:
            f.write(f"# oracle RIR, written by tests/golden/make_golden.py (oracle only)\n")
            f.write(f"# arXiv 2104.13347 Sec. II.A; params: {p}\n")
            f.write(f"# stats: {st}\n")
            for v in h:
                f.write(f"{v:.17g}\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
