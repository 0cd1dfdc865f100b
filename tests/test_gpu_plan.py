"""Plans: the dataset step of a fixed batch shape captured into CUDA graphs
and replayed (GPU).

A plan's runs must give, bit for bit, what the batch entry points give on
the same rooms (ism_rir_batch_ex at the plan's window, then
ism_convolve_batch with the same seed and noise ids): the graphs hold the
same kernels with the same launch shapes, and only the descriptors change
from run to run.  Runs alternate between two staging buffers, so three runs
with different rooms exercise both graphs and the reuse of the first.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def direct_step(ism, rooms, srcs, snr, base, seed, precision, window):
    import torch
    h = ism.rir_batch(rooms, window=window)
    M = [np.asarray(r["mics"]).reshape(-1, 3).shape[0] for r in rooms]
    jobs, ylen = ism.conv_jobs(M, [r["rir_len"] for r in rooms], [len(s) for s in srcs],
                               snr_db=snr, noise_ids=[base + i for i in range(len(rooms))])
    y = torch.empty(ylen, device="cuda")
    ism.convolve_batch(jobs, h, torch.from_numpy(np.concatenate(srcs)).cuda(), y, seed=seed,
                       precision=precision)
    torch.cuda.synchronize()
    return h, y


@pytest.mark.parametrize("precision", [0, 1])
def test_plan_runs_match_the_batch_entry_points(ism, precision):
    import torch
    n, W, seed = 6, 512, 4242
    shapes = dict(order=5, rir_len=2500, n_mics=5)
    sets = [wl.room_batch(n, seed=300 + k, **shapes) for k in range(3)]
    srcs = wl.sources(sets[0], 0.2, seed=310)
    lens = [len(s) for s in srcs]
    src = torch.from_numpy(np.concatenate(srcs)).cuda()
    n_rirs, hl = ism.rir_batch_size(sets[0])
    ylen = sum(5 * (L + 2499) for L in lens)
    h = torch.empty(hl, device="cuda")
    y = torch.empty(ylen, device="cuda")
    snr = [5.0, math.nan, 12.0, 30.0, math.nan, 0.0]
    with ism.Plan(sets[0], h, src, y, src_lens=lens, precision=precision, window=W,
                  max_order=6, seed=seed) as plan:
        for k, rooms in enumerate(sets):
            plan.run(rooms, snr_db=snr, noise_id_base=100 * k)
            torch.cuda.synchronize()
            hd, yd = direct_step(ism, rooms, srcs, snr, 100 * k, seed, precision, W)
            assert torch.equal(h, hd), k
            assert torch.equal(y, yd), k
        # the last run against the oracle (noise-free rooms 1 and 4)
        ref_h, _ = oracle.rir_batch(sets[2][:2])
        hv = h.view(n, 5, 2500).cpu().numpy().astype(np.float64)
        for m in range(5):
            assert rel_l2(hv[1, m], ref_h[1][m]) <= 1e-5
        yv = y.cpu().numpy().astype(np.float64)
        off = 5 * (lens[0] + 2499)
        T = lens[1] + 2499
        yref = oracle.convolve_batch([hv[1]], [srcs[1].astype(np.float64)])[0]
        for m in range(5):
            assert rel_l2(yv[off + m * T:off + (m + 1) * T], yref[m]) <= 1e-5


def test_plan_of_rirs_only_and_shape_checks(ism):
    import torch
    rooms = wl.single_room(seed=1001)
    h = torch.empty(4096, device="cuda")
    with ism.Plan(rooms, h, window=64) as plan:
        for seed in (1001, 1002, 1003):
            r = wl.single_room(seed=seed)
            plan.run(r)
            torch.cuda.synchronize()
            assert torch.equal(h, ism.rir_batch(r, window=64))
        bad = wl.single_room(seed=1004, rir_len=2048)
        with pytest.raises(ism.IsmError) as ei:
            plan.run(bad)
        assert ei.value.status == 2
        deep = wl.single_room(seed=1004, order=11)
        with pytest.raises(ism.IsmError) as ei:
            plan.run(deep)
        assert ei.value.status == 2


def test_plan_with_every_launch_group(ism):
    """A plan whose batch holds Hann-sinc RIRs, Lagrange RIRs and Hann RIRs
    that end before their direct arrival (the three launch groups of a RIR
    call, the last on the direct kernel), delay-limited orders with a
    capacity, and FP32 convolution: runs with new geometry match the batch
    entry points bit for bit."""
    import torch

    def batch(seed):
        rng = np.random.default_rng(seed)
        out = []
        for i in range(4):
            kind = i % 2
            r = wl.room_batch(1, seed=seed * 10 + i, order=-1, rir_len=700 + 300 * i, n_mics=3,
                              n_taps=8 if kind else 81, fd_kind=kind)[0]
            out.append(r)
        # a 24-sample RIR of mics about 1 m from the source (direct delay
        # ~47 samples): only the direct path's filter tail lands in it
        dx = 0.01 * rng.random()
        out.append(dict(dims=np.array([6.0, 5.0, 3.0]), beta=np.full(6, 0.8),
                        src=np.array([1.0 + dx, 1.0, 1.5]),
                        mics=np.array([[2.0, 1.0, 1.5], [1.0, 2.1, 1.5]]), fs=16000.0,
                        c=343.0, order=3, n_taps=81, fd_kind=0, rir_len=24))
        return out

    sets = [batch(500 + k) for k in range(3)]
    srcs = wl.sources(sets[0], 0.05, seed=510)
    lens = [len(s) for s in srcs]
    src = torch.from_numpy(np.concatenate(srcs)).cuda()
    _, hl = ism.rir_batch_size(sets[0])
    M = [len(r["mics"]) for r in sets[0]]
    ylen = sum(m * (T + r["rir_len"] - 1) for m, T, r in zip(M, lens, sets[0]))
    h = torch.empty(hl, device="cuda")
    y = torch.empty(ylen, device="cuda")
    with ism.Plan(sets[0], h, src, y, src_lens=lens, precision=ism.F32, window=256,
                  max_order=40, seed=3) as plan:
        for k, rooms in enumerate(sets):
            plan.run(rooms, snr_db=[10.0] * len(rooms), noise_id_base=7 * k)
            torch.cuda.synchronize()
            hd, yd = direct_step(ism, rooms, srcs, [10.0] * len(rooms), 7 * k, 3, ism.F32, 256)
            assert torch.equal(h, hd), k
            assert torch.equal(y, yd), k
