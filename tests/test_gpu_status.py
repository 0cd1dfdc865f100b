"""Kernel-reported errors reach the caller (GPU).

The split-BF16 convolution kernels bound every wait inside them; a wait
that runs out makes the kernel stop, write zeros for what it did not finish
and set the call's status cell.  These tests make a wait run out on purpose
through the library's injection switch (the MMA issuer waits, before issuing
anything, on a barrier nothing arrives at, with a 20 ms limit): a wait that
nothing ends, bounded, so the kernel returns and the context stays usable.
Each checks that the failure is reported as ISM_ERR_INTERNAL where the
header promises it, and that the next call runs clean and matches the oracle.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def conv_case(ism, L=2000, M=3, T=3000, seed=5):
    import torch
    rng = np.random.default_rng(seed)
    h = (rng.standard_normal((M, L)) * np.exp(-np.arange(L) / 500)).astype(np.float32)
    s = rng.standard_normal(T).astype(np.float32)
    jobs, ylen = ism.conv_jobs([M], [L], [T])
    return (h, s, jobs, torch.from_numpy(h.ravel()).cuda(), torch.from_numpy(s).cuda(),
            torch.full((ylen,), float("nan"), device="cuda"))


@pytest.mark.parametrize("L,T", [(2000, 3000), (30000, 26000)])  # one / two segment windows
def test_injected_timeout_reported_then_clean_call(ism, L, T):
    import torch
    h, s, jobs, hd, sd, y = conv_case(ism, L=L, T=T)
    stream = torch.cuda.current_stream()
    ism.debug_inject(ism.INJECT_CONV_WAIT)
    ism.convolve_batch(jobs, hd, sd, y, precision=ism.BF16X3)  # enqueued: OK
    with pytest.raises(ism.IsmError) as ei:
        ism.stream_status(stream)
    assert ei.value.status == 7  # ISM_ERR_INTERNAL
    yv = y.cpu().numpy()
    assert np.isfinite(yv).all() and not yv.any()  # the stopped kernel wrote zeros
    ism.stream_status(stream)  # reported once
    # the next call runs clean
    ism.convolve_batch(jobs, hd, sd, y, precision=ism.BF16X3)
    ism.stream_status(stream)
    ref = oracle.convolve_batch([h.astype(np.float64)], [s.astype(np.float64)])[0]
    got = y.cpu().numpy().astype(np.float64).reshape(ref.shape)
    for m in range(ref.shape[0]):
        assert rel_l2(got[m], ref[m]) <= 1e-5


def test_next_call_on_the_stream_reports_it(ism):
    import torch
    _, _, jobs, hd, sd, y = conv_case(ism)
    ism.debug_inject(ism.INJECT_CONV_WAIT)
    ism.convolve_batch(jobs, hd, sd, y, precision=ism.BF16X3)
    torch.cuda.synchronize()
    with pytest.raises(ism.IsmError) as ei:  # launches nothing
        ism.convolve_batch(jobs, hd, sd, y, precision=ism.BF16X3)
    assert ei.value.status == 7
    ism.convolve_batch(jobs, hd, sd, y, precision=ism.BF16X3)
    ism.stream_status()


def test_dataset_batch_reports_it(ism):
    import torch
    rooms = wl.room_batch(3, seed=61, order=3, rir_len=1000, n_mics=2)
    srcs = wl.sources(rooms, 0.1, seed=62)
    lens = [len(x) for x in srcs]
    src = torch.from_numpy(np.concatenate(srcs)).pin_memory()
    y = torch.empty(sum(2 * (T + 999) for T in lens), dtype=torch.float32).pin_memory()
    ism.debug_inject(ism.INJECT_CONV_WAIT)
    with pytest.raises(ism.IsmError) as ei:
        ism.dataset_batch(rooms, src, lens, y, precision=ism.BF16X3, chunk_rooms=3)
    assert ei.value.status == 7
    ism.dataset_batch(rooms, src, lens, y, precision=ism.BF16X3, chunk_rooms=3)
    assert torch.isfinite(y).all() and y.abs().sum() > 0


def test_served_batch_reports_it(ism):
    room = wl.room_batch(1, seed=63, order=3, rir_len=800, n_mics=2)[0]
    src = np.random.default_rng(64).standard_normal(1200).astype(np.float32)
    with ism.Server(precision=ism.BF16X3, n_streams=1) as srv:
        srv.wait(srv.submit(room, src), 60.0)  # warm: the server's first batch
        ism.debug_inject(ism.INJECT_CONV_WAIT)
        t = srv.submit(room, src)
        with pytest.raises(ism.IsmError) as ei:
            srv.wait(t, 60.0)
        assert ei.value.status == 7
        srv.release(t)
        t2 = srv.submit(room, src)
        res = srv.wait(t2, 60.0)
        assert res.n_mics == 2
        srv.release(t2)


def test_served_batch_allocation_failure(ism):
    """A failing device allocation in the server's admission path (injected:
    the allocator is not called) fails that batch's requests with
    ISM_ERR_OUT_OF_MEMORY and returns their budget; later requests run."""
    import time
    room = wl.room_batch(1, seed=65, order=3, rir_len=900, n_mics=3)[0]
    src = np.random.default_rng(66).standard_normal(1500).astype(np.float32)
    with ism.Server(precision=ism.F32, n_streams=1, max_batch=4) as srv:
        t0 = srv.submit(room, src)
        srv.wait(t0, 60.0)
        srv.release(t0)
        ism.debug_inject(ism.INJECT_SERVE_ALLOC)
        t = srv.submit(room, src)
        with pytest.raises(ism.IsmError) as ei:
            srv.wait(t, 60.0)
        assert ei.value.status == 3  # ISM_ERR_OUT_OF_MEMORY
        srv.release(t)
        t2 = srv.submit(room, src)
        res = srv.wait(t2, 60.0)
        assert res.n_mics == 3
        srv.release(t2)
        for _ in range(100):  # the server thread frees released batches
            if srv.stats()["bytes_in_use"] == 0:
                break
            time.sleep(0.01)
        st = srv.stats()
        assert st["bytes_in_use"] == 0 and st["completed"] >= 2
