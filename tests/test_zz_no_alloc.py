"""ism_rir_batch_noalloc against ism_rir_batch.

The no-alloc entry point serves callers that cannot allocate device memory
while they run (their memory is owned by another allocator, or they run in a
latency-bound loop where cudaMalloc is not acceptable).  It must give the
RIRs that the allocating entry point gives, on repeated calls that reuse its
fixed scratch.  This file is collected last so that a failure here comes
after every other test has run; it also passes on its own in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5  # rel-L2 per RIR, the FP32 RIR bar of the other GPU tests


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def test_noalloc_matches_allocating_entry_point(ism):
    import torch
    from paper_2104_13347_gb300 import _lib

    rooms = (wl.room_batch(6, seed=77, order=6, rir_len=3000, n_mics=4)
             + wl.room_batch(2, seed=78, order=5, rir_len=2100, n_mics=3, n_taps=8,
                             fd_kind=wl.FD_LAGRANGE))
    n_rirs, hl = ism.rir_batch_size(rooms)
    ref = ism.rir_batch(rooms)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy().astype(np.float64)
    lib = _lib.load()
    arr, keep = _lib.make_rooms(rooms)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((hl,), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.ism_rir_batch_noalloc(arr, len(rooms), ctypes.c_void_p(out.data_ptr()), None,
                                       stream)
        assert st == _lib.ISM_OK, _lib.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        o = 0
        for r in rooms:
            M = np.asarray(r["mics"]).shape[0]
            for m in range(M):
                seg = slice(o, o + r["rir_len"])
                assert rel_l2(got[seg], ref[seg]) <= TOL, f"call {call}, RIR at {o}"
                o += r["rir_len"]
        assert o == hl


def test_noalloc_explicit_offsets_through_the_binding(ism):
    """Per-RIR offsets (RIRs in reverse order, gaps between them) through the
    Python wrapper, against the allocating entry point given the same
    offsets; the gaps keep the caller's NaN fill."""
    import torch

    rooms = wl.room_batch(3, seed=80, order=5, rir_len=1500, n_mics=3)
    n_rirs, _ = ism.rir_batch_size(rooms)
    L, gap = 1500, 37
    offs = [(n_rirs - 1 - j) * (L + gap) + gap for j in range(n_rirs)]
    total = n_rirs * (L + gap) + gap
    ref = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    ism.rir_batch(rooms, h=ref, h_offsets=offs)
    prep = ism.PreparedRooms(rooms)
    for call in range(2):
        got = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
        ism.rir_batch_noalloc(prep if call else rooms, got, h_offsets=offs)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        filled = np.zeros(total, bool)
        for o in offs:
            filled[o:o + L] = True
            assert rel_l2(g[o:o + L], r[o:o + L]) <= TOL, f"call {call}, RIR at {o}"
        assert np.isnan(g[~filled]).all()
    end = max(o + L for o in offs)  # one float short of the farthest RIR's end
    with pytest.raises(ValueError):
        ism.rir_batch_noalloc(rooms, torch.empty(end - 1, device="cuda"), h_offsets=offs)


def test_noalloc_rejects_more_rirs_than_its_scratch(ism):
    import torch
    from paper_2104_13347_gb300 import _lib

    room = wl.room_batch(1, seed=79, order=1, rir_len=64,
                         n_mics=14561)[0]
    arr, keep = _lib.make_rooms([room])
    # a real buffer that holds the whole batch: a regression of the size
    # check shows up as a wrong status, not as writes to a bad address
    h = torch.zeros(14561 * 64, dtype=torch.float32, device="cuda")
    st = _lib.load().ism_rir_batch_noalloc(arr, 1, ctypes.c_void_p(h.data_ptr()), None, None)
    torch.cuda.synchronize()
    assert st == _lib.ISM_ERR_INVALID_ARG
    assert "14560" in _lib.last_error()
    assert not h.any().item()
