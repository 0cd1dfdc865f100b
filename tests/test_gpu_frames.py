"""Training frames on the GPU (ism_frames_batch; Sec. II.B: 1024-sample
multichannel windows of the convolved signals, Sec. III.A: measurement
noise at a drawn SNR) against the FP64 oracle.

Bars: clean frames bit-exact copies (zero padded outside the signal);
noisy frames within 1e-5 of the oracle relative to sigma (the Gaussian is
evaluated in FP32 on the GPU) and sigma within 1e-6 relative."""
import math

import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_frames_against_oracle(ism):
    import torch
    rng = np.random.default_rng(17)
    # three "rooms" of convolved signals of different sizes, packed
    shapes = [(7, 3000), (4, 1500), (1, 900)]
    ys = [rng.standard_normal(s).astype(np.float32) * rng.uniform(0.1, 2.0) for s in shapes]
    offs = np.cumsum([0] + [a * b for a, b in shapes])[:-1]
    y = torch.from_numpy(np.concatenate([a.ravel() for a in ys])).cuda()
    frame_len = 256
    picks, t0s, snrs = [], [], []
    for i in range(60):
        r = int(rng.integers(3))
        picks.append(r)
        t0s.append(int(rng.integers(-300, shapes[r][1] + 50)))
        snrs.append([math.inf, math.nan, float(rng.uniform(0, 40))][i % 3])
    jobs, n_out = ism.frame_jobs([offs[r] for r in picks], [shapes[r][1] for r in picks],
                                 [shapes[r][0] for r in picks], t0s, frame_len, snr_db=snrs,
                                 noise_ids=[1000 + i for i in range(60)])
    out = torch.full((n_out,), float("nan"), device="cuda")
    ism.frames_batch(jobs, frame_len, y, out, seed=99)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    for i, r in enumerate(picks):
        M = shapes[r][0]
        g = got[jobs[i].out_offset:jobs[i].out_offset + M * frame_len].reshape(M, frame_len)
        ref, sig = oracle.frame(ys[r].astype(np.float64), t0s[i], frame_len, snrs[i], 99, 1000 + i)
        if sig == 0.0:
            np.testing.assert_array_equal(g, ref)
        else:
            assert np.max(np.abs(g - ref)) <= 1e-5 * sig + 1e-6 * np.max(np.abs(ref))


def test_frames_from_convolved_rooms(ism):
    """End to end: RIRs, clean convolution, then 1024-sample training frames
    at SNR >= 20 dB (the paper's augmentation range) from random rooms and
    offsets; frames equal the oracle frames of the same clean signals."""
    import torch
    rooms = wl.room_batch(4, seed=77, order=6, rir_len=2048)
    h = ism.rir_batch(rooms)
    srcs = wl.sources(rooms, 0.3, seed=78)
    jobs, ylen = ism.conv_jobs([8] * 4, [2048] * 4, [len(s) for s in srcs])
    y = torch.empty(ylen, device="cuda")
    ism.convolve_batch(jobs, h, torch.from_numpy(np.concatenate(srcs)).cuda(), y, precision=1)
    T = len(srcs[0]) + 2048 - 1
    rng = np.random.default_rng(5)
    n = 32
    rr = rng.integers(0, 4, n)
    t0s = rng.integers(0, T - 1024, n)
    snrs = 20.0 + rng.exponential(10.0, n)
    fj, n_out = ism.frame_jobs([int(r) * 8 * T for r in rr], [T] * n, [8] * n, t0s, 1024,
                               snr_db=snrs)
    out = torch.empty(n_out, device="cuda")
    ism.frames_batch(fj, 1024, y, out, seed=5)
    torch.cuda.synchronize()
    yy = y.cpu().numpy().astype(np.float64).reshape(4, 8, T)
    got = out.cpu().numpy().astype(np.float64).reshape(n, 8, 1024)
    for i in range(n):
        ref, sig = oracle.frame(yy[rr[i]], int(t0s[i]), 1024, float(snrs[i]), 5, i)
        assert np.max(np.abs(got[i] - ref)) <= 1e-5 * sig + 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("frame_len,mics", [(333, 5), (1024, 8), (1023, 3), (1, 7),
                                            (2000, 2), (512, 12)])
def test_frames_shapes_and_alignments(ism, frame_len, mics):
    """Frame lengths and mic counts on both kernels (frames of at most 1024
    samples and 8 mics are held in registers between the two passes, longer
    frames or more mics take the two-pass kernel), rows of odd length from an
    odd offset and frames packed at odd offsets, so that 8-byte and 4-byte
    accesses both occur, and frames reaching past either end of the signal;
    against the oracle frame by frame."""
    import torch
    rng = np.random.default_rng(1000 * frame_len + mics)
    T, base, n_rooms = 2501, 3, 3
    ys = [rng.standard_normal((mics, T)) * rng.uniform(0.2, 3.0) for _ in range(n_rooms)]
    buf = np.concatenate([np.zeros(base)] + [a.ravel() for a in ys]).astype(np.float32)
    ys = [a.astype(np.float32).astype(np.float64) for a in ys]
    y = torch.from_numpy(buf).cuda()
    n = 40
    rr = rng.integers(0, n_rooms, n)
    t0s = rng.integers(-frame_len - 5, T + 5, n)
    snrs = [[math.inf, math.nan, float(rng.uniform(-10, 40))][i % 3] for i in range(n)]
    jobs, n_out = ism.frame_jobs([base + int(r) * mics * T for r in rr], [T] * n, [mics] * n,
                                 t0s, frame_len, snr_db=snrs, noise_ids=[77 + i for i in range(n)])
    out = torch.full((n_out,), float("nan"), device="cuda")
    ism.frames_batch(jobs, frame_len, y, out, seed=31)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    for i in range(n):
        g = got[jobs[i].out_offset:jobs[i].out_offset + mics * frame_len].reshape(mics, frame_len)
        ref, sig = oracle.frame(ys[rr[i]], int(t0s[i]), frame_len, snrs[i], 31, 77 + i)
        if sig == 0.0:
            np.testing.assert_array_equal(g, ref)
        else:
            assert np.max(np.abs(g - ref)) <= 1e-5 * sig + 1e-6 * np.max(np.abs(ref)), i
