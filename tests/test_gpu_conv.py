"""GPU parity of the convolution (K2b FP32 direct; K2 split-BF16 tensor
cores) and the noise epilogue against the FP64 oracle (arXiv 2104.13347,
Sec. II.A batch convolution; Sec. III.A noise at a chosen SNR).

Bars: rel-L2 <= 1e-5 per (room, mic) for both the FP32 path and the
split-BF16 path (which measures ~5e-6 on the 1024-room batch, well inside the
2e-4 that a split-BF16 convolution is allowed);
noise uniforms exactly the oracle's, Gaussian values within 1e-5 absolute,
sigma within 1e-6 relative of the oracle's sigma on the same clean signal.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-5}
# Outputs that sum over tens of thousands of taps: the split-BF16 error grows
# with the number of terms (the three products accumulate in one FP32
# tensor-core accumulator), so these cases take the 2e-4 bar the
# specification sets for the split-BF16 convolution (measured 2.3e-5 for
# 22.5k flat random taps against 27k source samples); FP32 keeps 1e-5.
TOL_LONG = {0: 1e-5, 1: 2e-4}


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def run_conv(ism, hs, srcs, precision, snr=None, seed=0, noise_ids=None):
    import torch
    jobs, ylen = ism.conv_jobs([h.shape[0] for h in hs], [h.shape[1] for h in hs],
                               [len(s) for s in srcs], snr_db=snr, noise_ids=noise_ids)
    hcat = torch.from_numpy(np.concatenate([h.ravel() for h in hs]).astype(np.float32)).cuda()
    scat = torch.from_numpy(np.concatenate(srcs).astype(np.float32)).cuda()
    y = torch.full((ylen,), float("nan"), device="cuda")
    ism.convolve_batch(jobs, hcat, scat, y, seed=seed, precision=precision)
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    out, o = [], 0
    for h, s in zip(hs, srcs):
        T = len(s) + h.shape[1] - 1
        out.append(y[o:o + h.shape[0] * T].reshape(h.shape[0], T))
        o += h.shape[0] * T
    return out


def ragged_case(seed=3):
    rng = np.random.default_rng(seed)
    hs, ss = [], []
    for i in range(6):
        M = int(rng.integers(1, 12))
        L = int(rng.integers(1, 3000))
        T = int(rng.integers(1, 5000))
        hs.append((rng.standard_normal((M, L)) * np.exp(-np.arange(L) / 800)).astype(np.float32))
        ss.append(rng.standard_normal(T).astype(np.float32))
    return hs, ss


@pytest.mark.parametrize("precision", [0, 1])
def test_conv_ragged_parity(ism, precision):
    hs, ss = ragged_case()
    got = run_conv(ism, hs, ss, precision)
    ref = oracle.convolve_batch([h.astype(np.float64) for h in hs],
                                [s.astype(np.float64) for s in ss])
    for g, r in zip(got, ref):
        assert g.shape == r.shape
        for m in range(g.shape[0]):
            assert rel_l2(g[m], r[m]) <= TOL[precision]


def test_conv_delta_rir_bf16x3(ism):
    """A delta RIR is exact in bf16 (lo = 0), so the split path returns the
    source to the split's representation error (2^-16 relative)."""
    rng = np.random.default_rng(8)
    s = rng.standard_normal(3000).astype(np.float32)
    h = np.zeros((2, 700), np.float32)
    h[0, 0] = 1.0
    h[1, 613] = 1.0
    (y,) = run_conv(ism, [h], [s], 1)
    np.testing.assert_allclose(y[0, :3000], s, rtol=2e-5, atol=0)
    assert not np.any(y[0, 3000:])
    np.testing.assert_allclose(y[1, 613:3613], s, rtol=2e-5, atol=0)
    assert not np.any(y[1, :613])


def test_conv_long_rir_and_many_mics(ism):
    """RIR longer than a tile and 11 mics (two mic groups), both paths."""
    rng = np.random.default_rng(12)
    hs = [(rng.standard_normal((11, 5000)) * np.exp(-np.arange(5000) / 1500)).astype(np.float32)]
    ss = [rng.standard_normal(2500).astype(np.float32)]
    ref = oracle.convolve_batch([hs[0].astype(np.float64)], [ss[0].astype(np.float64)])[0]
    for precision in (0, 1):
        (y,) = run_conv(ism, hs, ss, precision)
        for m in range(11):
            assert rel_l2(y[m], ref[m]) <= TOL[precision]


def test_conv_segment_boundary(ism):
    """The persistent three-product kernel cuts a tile's live 64-tap chunks
    into segment windows of 352 chunks: RIRs of 22513 samples (352 chunks,
    one window) and 22514 (353, two) with sources long enough that middle
    tiles have every chunk live, a 50001-sample RIR (several windows per
    tile) and a 9-mic room (a partial 8-mic group), both precisions, against
    the oracle; each room's result is the same, bit for bit, when it is
    convolved alone."""
    rng = np.random.default_rng(21)
    lens, mics, srcl = (22513, 22514, 50001, 37), (2, 3, 1, 9), (27000, 27100, 30000, 4100)
    hs = [(rng.standard_normal((M, L)) * np.exp(-np.arange(L) / 6000)).astype(np.float32)
          for M, L in zip(mics, lens)]
    ss = [rng.standard_normal(T).astype(np.float32) for T in srcl]
    ref = oracle.convolve_batch([h.astype(np.float64) for h in hs],
                                [s.astype(np.float64) for s in ss])
    for precision in (0, 1):
        got = run_conv(ism, hs, ss, precision)
        for i, (g, r) in enumerate(zip(got, ref)):
            assert g.shape == r.shape
            for m in range(g.shape[0]):
                assert rel_l2(g[m], r[m]) <= TOL_LONG[precision], (precision, i, m)
            (alone,) = run_conv(ism, [hs[i]], [ss[i]], precision)
            np.testing.assert_array_equal(alone, g)


@pytest.mark.parametrize("precision", [0, 1])
def test_conv_degenerate_sizes(ism, precision):
    """1-sample RIRs and sources, one mic and nine mics (a partial 8-mic
    group), in one batch: each (room, mic) within the bar of the oracle."""
    rng = np.random.default_rng(31)
    shapes = [(1, 1, 1), (1, 1, 5000), (2, 3000, 1), (9, 1, 2), (9, 700, 3), (1, 4097, 4095)]
    hs = [(rng.standard_normal((M, L)) + 0.5).astype(np.float32) for M, L, _ in shapes]
    ss = [(rng.standard_normal(T) + 0.25).astype(np.float32) for _, _, T in shapes]
    got = run_conv(ism, hs, ss, precision)
    ref = oracle.convolve_batch([h.astype(np.float64) for h in hs],
                                [s.astype(np.float64) for s in ss])
    for i, (g, r) in enumerate(zip(got, ref)):
        assert g.shape == r.shape, i
        for m in range(g.shape[0]):
            assert rel_l2(g[m], r[m]) <= TOL[precision], (i, m)


def test_conv_short_and_long_rirs_in_one_call(ism):
    """RIRs of 2000, 30000 and 40000 samples in one split-BF16 call (the
    persistent kernel, the longer two in several segment windows per tile
    where the source covers enough chunks), against the oracle."""
    rng = np.random.default_rng(32)
    lens, mics, srcl = (2000, 30000, 40000), (3, 2, 2), (6000, 24000, 2500)
    hs = [(rng.standard_normal((M, L)) * np.exp(-np.arange(L) / 4000)).astype(np.float32)
          for M, L in zip(mics, lens)]
    ss = [rng.standard_normal(T).astype(np.float32) for T in srcl]
    got = run_conv(ism, hs, ss, 1)
    ref = oracle.convolve_batch([h.astype(np.float64) for h in hs],
                                [s.astype(np.float64) for s in ss])
    for i, (g, r) in enumerate(zip(got, ref)):
        for m in range(g.shape[0]):
            assert rel_l2(g[m], r[m]) <= TOL_LONG[1], (i, m)


def test_conv_delta_rir_exact(ism):
    rng = np.random.default_rng(8)
    s = rng.standard_normal(3000).astype(np.float32)
    h = np.zeros((2, 700), np.float32)
    h[0, 0] = 1.0
    h[1, 613] = 1.0
    (y,) = run_conv(ism, [h], [s], 0)
    np.testing.assert_array_equal(y[0, :3000], s)
    assert not np.any(y[0, 3000:])
    np.testing.assert_array_equal(y[1, 613:3613], s)


def test_noise_matches_oracle(ism):
    hs, ss = ragged_case(seed=9)
    snr = np.linspace(0, 30, len(hs)).astype(np.float32)
    ids = [1000 + 7 * i for i in range(len(hs))]
    clean = run_conv(ism, hs, ss, 0)
    noisy = run_conv(ism, hs, ss, 0, snr=snr, seed=1234, noise_ids=ids)
    for i, (c, n) in enumerate(zip(clean, noisy)):
        d = n - c
        p_sig = np.mean(c ** 2)
        sigma = math.sqrt(p_sig / 10 ** (snr[i] / 10))
        M, T = c.shape
        rng = np.random.default_rng(i)
        for _ in range(20):
            m, t = int(rng.integers(M)), int(rng.integers(T))
            z = oracle.gauss(1234, ids[i], m, t)
            assert abs(d[m, t] - sigma * z) <= 1e-5 * sigma * (1 + abs(z)) + 2e-6 * abs(c[m, t])
        if d.size > 1000:
            assert abs(10 * np.log10(p_sig / np.mean(d ** 2)) - snr[i]) < 0.5


def test_noise_dense_against_oracle(ism):
    """Every sample of a long noisy 8-mic signal against the oracle's noise
    (Sec. III.A): the deviates within 2e-6 (1 + |z|) of the oracle's
    (measured 9.6e-7), plus the FP32 rounding of y + sigma z.  4.2e6 draws
    reach u1 within 2^-6 of 1 (the series branch of the logarithm) ~6e4
    times and every octant of the Box--Muller angle."""
    rng = np.random.default_rng(77)
    h = (rng.standard_normal((8, 64)) * np.exp(-np.arange(64) / 16)).astype(np.float32)
    s = rng.standard_normal(1 << 20).astype(np.float32)
    (clean,) = run_conv(ism, [h], [s], 0)
    (noisy,) = run_conv(ism, [h], [s], 0, snr=np.array([12.5], np.float32), seed=4321,
                        noise_ids=[4242])
    ref, sigma = oracle.add_noise(clean.copy(), 12.5, 4321, 4242)
    z = (ref - clean) / sigma
    err = np.abs(noisy - ref)
    bar = 2e-6 * sigma * (1 + np.abs(z)) + 2.0 ** -22 * np.abs(clean)
    assert np.all(err <= bar), float(np.max(err / bar))


def test_noise_split_bf16_against_oracle(ism):
    """The noise level of the split-BF16 path comes from the y^2 sums of the
    tensor-core kernel's epilogue (FP32 within a 32-column block, float-float
    across blocks, FP64 across rows and tiles); sigma and every noise value
    against the oracle's (Sec. III.A) on the kernel's own noise-free output:
    ragged rooms, a 9-mic room (a partial 8-mic group) and a room of 7
    output tiles whose last block the signal's end cuts."""
    hs, ss = ragged_case(seed=19)
    rng = np.random.default_rng(23)
    hs.append((rng.standard_normal((9, 700)) * np.exp(-np.arange(700) / 200)).astype(np.float32))
    ss.append(rng.standard_normal(2100).astype(np.float32))
    hs.append((rng.standard_normal((8, 5000)) * np.exp(-np.arange(5000) / 900)).astype(np.float32))
    ss.append(rng.standard_normal(20000).astype(np.float32))
    snr = np.linspace(2, 28, len(hs)).astype(np.float32)
    ids = [3000 + 11 * i for i in range(len(hs))]
    clean = run_conv(ism, hs, ss, 1)
    noisy = run_conv(ism, hs, ss, 1, snr=snr, seed=2468, noise_ids=ids)
    for i, (c, n) in enumerate(zip(clean, noisy)):
        ref, sigma = oracle.add_noise(c.copy(), float(snr[i]), 2468, ids[i])
        z = (ref - c) / sigma
        bar = 2e-6 * sigma * (1 + np.abs(z)) + 2.0 ** -22 * np.abs(c)
        assert np.all(np.abs(n - ref) <= bar), (i, float(np.max(np.abs(n - ref) / bar)))


@pytest.mark.parametrize("precision", [0, 1])
def test_noise_degenerate_levels(ism, precision):
    """Noise levels at the edges of Sec. III.A's augmentation, in one call:
    a silent room (zero source: mean power 0, so sigma = 0 and the output
    stays exactly zero -- u1 never reaches 0, so no deviate is infinite), a
    room with SNR NaN (no noise: bitwise the noise-free output), noise 20 dB
    above the signal, noise 80 dB below it, and an ordinary room with a
    9-mic array; each against the oracle's noise on the kernel's own
    noise-free output."""
    rng = np.random.default_rng(91)
    shapes = [(3, 900), (2, 400), (9, 1200), (4, 50), (8, 2000)]
    hs = [(rng.standard_normal((M, L)) * np.exp(-np.arange(L) / 300)).astype(np.float32)
          for M, L in shapes]
    ss = [np.zeros(1500, np.float32)] + [rng.standard_normal(T).astype(np.float32)
                                         for T in (700, 3000, 64, 5000)]
    snr = np.array([10.0, np.nan, -20.0, 80.0, 7.5], np.float32)
    ids = [901, 902, 903, 904, 905]
    clean = run_conv(ism, hs, ss, precision)
    noisy = run_conv(ism, hs, ss, precision, snr=snr, seed=97, noise_ids=ids)
    assert not np.any(clean[0]) and not np.any(noisy[0])
    np.testing.assert_array_equal(noisy[1], clean[1])
    for i in (2, 3, 4):
        ref, sigma = oracle.add_noise(clean[i].copy(), float(snr[i]), 97, ids[i])
        assert sigma > 0
        z = (ref - clean[i]) / sigma
        bar = 2e-6 * sigma * (1 + np.abs(z)) + 2.0 ** -22 * np.abs(clean[i])
        assert np.all(np.abs(noisy[i] - ref) <= bar), (i, float(np.max(np.abs(noisy[i] - ref) / bar)))


def test_noise_same_in_any_batch(ism):
    hs, ss = ragged_case(seed=10)
    snr = np.full(len(hs), 10.0, np.float32)
    ids = list(range(50, 50 + len(hs)))
    full = run_conv(ism, hs, ss, 0, snr=snr, seed=77, noise_ids=ids)
    part = run_conv(ism, hs[2:4], ss[2:4], 0, snr=snr[2:4], seed=77, noise_ids=ids[2:4])
    np.testing.assert_array_equal(full[2], part[0])
    np.testing.assert_array_equal(full[3], part[1])


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_conv_sampled(ism, precision):
    """1024 rooms x 8 mics, 8192-sample RIRs, 1 s sources at 16 kHz, in the
    benchmark's launch configuration; sampled outputs against the oracle."""
    import torch
    rooms = wl.room_batch(1024, seed=1002)
    h = ism.rir_batch(rooms)
    srcs = wl.sources(rooms, 1.0, seed=1003)
    jobs, ylen = ism.conv_jobs([8] * 1024, [8192] * 1024, [len(s) for s in srcs])
    scat = torch.from_numpy(np.concatenate(srcs)).cuda()
    y = torch.empty(ylen, device="cuda")
    ism.convolve_batch(jobs, h, scat, y, precision=precision)
    torch.cuda.synchronize()
    T = 16000 + 8192 - 1
    y = y.view(1024, 8, T)
    hv = h.view(1024, 8, 8192)
    rng = np.random.default_rng(2)
    for r in rng.choice(1024, 3, replace=False):
        m = int(rng.integers(8))
        ts = np.sort(rng.choice(T, 400, replace=False))
        ref = oracle.convolve_at(hv[r, m].cpu().numpy().astype(np.float64),
                                 srcs[r].astype(np.float64), ts)
        got = y[r, m].cpu().numpy().astype(np.float64)[ts]
        assert rel_l2(got, ref) <= TOL[precision]
    assert torch.isfinite(y).all()
