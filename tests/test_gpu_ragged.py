"""Ragged batches (RT60-driven RIR lengths, 16 and 48 kHz, 4-16 mics, order
from the length, Sabine wall coefficients) through the RIR and convolution
kernels, checked against the FP64 oracle (arXiv 2104.13347 Sec. II.A: the
paper keeps every reflection arriving within the reverberation time).
"""
import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def test_ragged_batch_rir_and_conv(ism):
    import torch
    # 40 requests of the ragged recipe, RT60 up to 0.35 s so that the oracle
    # finishes in seconds; every length, rate and mic count differs
    rooms = wl.ragged_batch(40, seed=1005, rt_hi=0.35)
    n_rirs, hl = ism.rir_batch_size(rooms)
    stats = torch.zeros(2 * n_rirs, dtype=torch.int64, device="cuda")
    h = ism.rir_batch(rooms, stats=stats)
    torch.cuda.synchronize()
    hh = h.cpu().numpy().astype(np.float64)
    st = stats.view(-1, 2).cpu().numpy()
    offs = np.cumsum([0] + [len(r["mics"]) * r["rir_len"] for r in rooms])
    rir0 = np.cumsum([0] + [len(r["mics"]) for r in rooms])
    rng = np.random.default_rng(1)
    picks = rng.choice(len(rooms), 5, replace=False)
    sub = [dict(rooms[i], mics=np.asarray(rooms[i]["mics"])[:1]) for i in picks]
    ref, ost = oracle.rir_batch(sub)
    for k, i in enumerate(picks):
        L = rooms[i]["rir_len"]
        got = hh[offs[i]:offs[i] + L]
        assert rel_l2(got, ref[k][0]) <= 1e-5
        assert st[rir0[i], 0] == ost[k, 1] and st[rir0[i], 1] == ost[k, 2]
    # convolution of each request's RIRs with its own source (0.25 s at its fs)
    srcs = wl.sources(rooms, 0.25, seed=7)
    jobs, ylen = ism.conv_jobs([len(r["mics"]) for r in rooms], [r["rir_len"] for r in rooms],
                               [len(s) for s in srcs])
    scat = torch.from_numpy(np.concatenate(srcs)).cuda()
    for precision in (0, 1):
        y = torch.empty(ylen, device="cuda")
        ism.convolve_batch(jobs, h, scat, y, precision=precision)
        torch.cuda.synchronize()
        yy = y.cpu().numpy().astype(np.float64)
        yo = 0
        for j, (r, s) in enumerate(zip(rooms, srcs)):
            M, L, T = len(r["mics"]), r["rir_len"], len(s)
            if j in picks[:3]:
                hj = hh[offs[j]:offs[j] + M * L].reshape(M, L)
                yr = oracle.convolve(hj[0], s.astype(np.float64))
                assert rel_l2(yy[yo:yo + T + L - 1], yr) <= 1e-5
            yo += M * (T + L - 1)


def test_long_rir_48k(ism):
    """One long 48 kHz RIR (RT60 0.9 s in a 19 x 17 x 16 m hall: 43200
    samples, order from the length) -- more windows than any other test --
    and its split-BF16 convolution through the persistent tensor-core kernel
    (a short source: one segment window per tile)."""
    import torch
    dims = np.array([19.0, 17.0, 16.0])
    rt60, fs = 0.9, 48000.0
    L = int(np.ceil(rt60 * fs))
    room = dict(dims=dims, beta=np.full(6, wl.sabine_beta(dims, rt60)),
                src=np.array([4.1, 11.3, 2.2]),
                mics=wl.circular_array(np.array([13.0, 6.0, 1.7]), 2, 0.05), fs=fs, c=343.0,
                order=wl.order_for_length(dims, L, fs, 343.0, 81), n_taps=81, fd_kind=0,
                rir_len=L)
    h = ism.rir_batch([room])
    torch.cuda.synchronize()
    assert L > 40000
    ref, _ = oracle.rir_batch([dict(room, mics=room["mics"][:1])])
    assert rel_l2(h[:L].cpu().numpy().astype(np.float64), ref[0][0]) <= 1e-5
    s = wl.sources([room], 0.1, seed=3)[0]
    jobs, ylen = ism.conv_jobs([2], [L], [len(s)])
    y = torch.empty(ylen, device="cuda")
    ism.convolve_batch(jobs, h, torch.from_numpy(s).cuda(), y, precision=1)
    torch.cuda.synchronize()
    ts = np.random.default_rng(4).choice(len(s) + L - 1, 300, replace=False)
    yr = oracle.convolve_at(h[:L].cpu().numpy().astype(np.float64), s.astype(np.float64), ts)
    assert rel_l2(y.cpu().numpy()[ts].astype(np.float64), yr) <= 1e-5
