"""The window autotuner of the image-source kernel (GPU).

A call with window = WINDOW_TUNE tunes its bucket on first use (each
candidate window timed on the call's stream), keeps the fastest, records it
in the ISM_TUNE_CACHE file, and leaves the outputs of the chosen window:
they match the FP64 oracle (arXiv 2104.13347 Sec. II.A RIRs) and are
bitwise those of a call with that window given explicitly, on every call.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


@pytest.mark.parametrize("kind,taps", [(0, 81), (1, 8)])
def test_tuned_window_parity_and_stability(ism, tmp_path, kind, taps):
    import torch
    cache = tmp_path / "tune.txt"
    os.environ["ISM_TUNE_CACHE"] = str(cache)
    try:
        rooms = wl.room_batch(40, seed=90 + kind, order=6, rir_len=3000, n_mics=4,
                              n_taps=taps, fd_kind=kind)
        assert ism.rir_tuned_window(rooms) == 0
        h1 = ism.rir_batch(rooms, window=ism.WINDOW_TUNE)
        torch.cuda.synchronize()
        W = ism.rir_tuned_window(rooms)
        assert W % 32 == 0 and 64 <= W <= 2048
        lines = cache.read_text().splitlines()
        assert len(lines) == 1 and lines[0].startswith("ism-tune 1 ")
        assert int(lines[0].split()[10]) == W
        h2 = ism.rir_batch(rooms, window=ism.WINDOW_TUNE)
        h3 = ism.rir_batch(rooms, window=W)
        torch.cuda.synchronize()
        assert torch.equal(h1, h2) and torch.equal(h1, h3)
        assert len(cache.read_text().splitlines()) == 1  # no second tuning
        ref, _ = oracle.rir_batch(rooms[:2])
        hv = h1.view(40, 4, 3000).cpu().numpy().astype(np.float64)
        for r in range(2):
            for m in range(4):
                assert rel_l2(hv[r, m], ref[r][m]) <= 1e-5
    finally:
        os.environ.pop("ISM_TUNE_CACHE", None)


def test_tuned_window_statistics_counted_once(ism):
    """Tuning runs the call several times; the statistics are those of one
    call."""
    import torch
    rooms = wl.room_batch(5, seed=95, order=4, rir_len=1500, n_mics=3)
    n_rirs, _ = ism.rir_batch_size(rooms)
    s1 = torch.zeros(2 * n_rirs, dtype=torch.int64, device="cuda")
    s2 = torch.zeros(2 * n_rirs, dtype=torch.int64, device="cuda")
    ism.rir_batch(rooms, window=ism.WINDOW_TUNE, stats=s1)
    ism.rir_batch(rooms, stats=s2)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)


def test_tuned_window_mixed_call(ism, tmp_path):
    """A call mixing both filters and RIR lengths tunes one window for the
    call; its RIRs are those of that window given explicitly."""
    import torch
    os.environ["ISM_TUNE_CACHE"] = str(tmp_path / "t.txt")
    try:
        rooms = (wl.room_batch(20, seed=97, order=5, rir_len=2500, n_mics=3)
                 + wl.room_batch(20, seed=98, order=4, rir_len=1200, n_mics=2, n_taps=8,
                                 fd_kind=wl.FD_LAGRANGE))
        h1 = ism.rir_batch(rooms, window=ism.WINDOW_TUNE)
        W = ism.rir_tuned_window(rooms)
        h2 = ism.rir_batch(rooms, window=W)
        torch.cuda.synchronize()
        assert W > 0 and torch.equal(h1, h2)
    finally:
        os.environ.pop("ISM_TUNE_CACHE", None)
