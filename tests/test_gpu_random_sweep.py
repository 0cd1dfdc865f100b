"""A seeded random sweep of the RIR, convolution and noise paths against
the FP64 oracle (Sec. II.A / III.A), beyond the hand-picked cases: batches
of 1-6 rooms of 0.6-20 m with wall coefficients anywhere in [0, 1] (0, 1
and 1e-20 included), sources and mics anywhere inside (some 1 mm from a
wall), 1-20 mics, lattice orders 0-6 or the delay-limited set, Hann
filters of 1-255 taps and Lagrange filters of 2-16, 8-192 kHz, speeds of
sound of 150, 343 and 1500 m/s and RIRs of 1-20000 samples.  Every batch
runs on the sparse path (automatic and a random window) and the direct
path (RIRs within 1e-5 rel-L2 of the oracle, image and tap counts exact),
then the convolution of the oracle's RIRs with random sources in both
precisions (1e-5 and the split-BF16 bar of 2e-4) and its noise at random
SNRs (NaN: none) against the oracle's noise on the kernel's own noise-free
output.  A second sweep sends random batches through the host-buffer
dataset step and the server and compares them with the batch entry points
bit for bit."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

N_BATCHES = 150


def draw_rooms(rng):
    rooms = []
    for _ in range(int(rng.integers(1, 7))):
        dims = rng.uniform(0.6, 20, 3) if rng.random() < 0.8 else rng.uniform(0.6, 3, 3)
        kind = 0 if rng.random() < 0.75 else 1
        taps = (int(rng.choice([1, 3, 9, 31, 81, 127, 255])) if kind == 0
                else int(rng.choice([2, 4, 8, 16])))
        fs = float(rng.choice([8000, 16000, 44100, 48000, 96000, 192000]))
        c = 343.0 if rng.random() < 0.85 else float(rng.choice([150.0, 1500.0]))
        beta = rng.uniform(0, 1, 6)
        beta[rng.random(6) < 0.1] = 0.0
        beta[rng.random(6) < 0.1] = 1.0
        beta[rng.random(6) < 0.05] = 1e-20

        def point():
            p = rng.uniform(0.05, 0.95, 3) * dims
            if rng.random() < 0.2:
                a = int(rng.integers(3))
                p[a] = 1e-3 if rng.random() < 0.5 else dims[a] - 1e-3
            return p

        src = point()
        n_m = int(rng.integers(1, 10)) if rng.random() < 0.85 else int(rng.integers(10, 21))
        mics = []
        while len(mics) < n_m:
            m = point()
            if np.linalg.norm(m - src) > 1e-3:
                mics.append(m)
        if rng.random() < 0.5:
            order, rir_len = int(rng.integers(0, 7)), int(rng.integers(1, 20001))
        else:
            # delay-limited set, at most ~4e4 images within reach
            order = -1
            reach = (3 * 4e4 * float(np.prod(dims)) / (4 * math.pi)) ** (1 / 3)
            rir_len = int(rng.integers(1, min(max(1, int(reach * fs / c) - taps), 20000) + 1))
        rooms.append(dict(dims=dims, beta=beta, src=src, mics=np.stack(mics), fs=fs, c=c,
                          order=order, n_taps=taps, fd_kind=kind, rir_len=rir_len))
    return rooms


def rel_l2(g, x):
    n = np.linalg.norm(x)
    if n == 0:
        return 0.0 if not np.any(g) else math.inf
    return float(np.linalg.norm(g - x) / n)


def test_random_rooms_against_oracle(ism):
    import torch
    rng = np.random.default_rng(2104)
    for b in range(N_BATCHES):
        rooms = draw_rooms(rng)
        ref, ost = oracle.rir_batch(rooms)
        n_rirs, _ = ism.rir_batch_size(rooms)
        for variant, window in ((0, 0), (1, 0), (0, 32 * int(rng.integers(1, 65)))):
            stats = torch.zeros(2 * n_rirs, dtype=torch.int64, device="cuda")
            h = ism.rir_batch(rooms, stats=stats, variant=variant, window=window)
            torch.cuda.synchronize()
            hh = h.cpu().numpy().astype(np.float64)
            st = stats.view(-1, 2).cpu().numpy()
            o = 0
            for ri, (r, rr) in enumerate(zip(rooms, ref)):
                for m in range(len(r["mics"])):
                    e = rel_l2(hh[o:o + r["rir_len"]], rr[m])
                    assert e <= 1e-5, (b, variant, window, ri, m, e, r)
                    o += r["rir_len"]
            np.testing.assert_array_equal(st[:, 0], ost[:, 1])
            np.testing.assert_array_equal(st[:, 1], ost[:, 2])
        ok = [i for i, r in enumerate(rooms) if r["rir_len"] <= 6000]
        if not ok:
            continue
        hs = [ref[i].astype(np.float32) for i in ok]
        ss = [rng.standard_normal(int(rng.integers(1, 4001))).astype(np.float32) for _ in ok]
        refc = oracle.convolve_batch([x.astype(np.float64) for x in hs],
                                     [s.astype(np.float64) for s in ss])
        snr = rng.uniform(-10, 60, len(ok)).astype(np.float32)
        snr[rng.random(len(ok)) < 0.2] = np.nan
        ids = [int(x) for x in rng.integers(0, 1 << 40, len(ok))]
        shape = ([x.shape[0] for x in hs], [x.shape[1] for x in hs], [len(s) for s in ss])
        jobs, ylen = ism.conv_jobs(*shape)
        jobs_n, _ = ism.conv_jobs(*shape, snr_db=snr, noise_ids=ids)
        hcat = torch.from_numpy(np.concatenate([x.ravel() for x in hs])).cuda()
        scat = torch.from_numpy(np.concatenate(ss)).cuda()
        for prec, tol in ((0, 1e-5), (1, 2e-4)):
            yc = torch.full((ylen,), float("nan"), device="cuda")
            yn = torch.full((ylen,), float("nan"), device="cuda")
            ism.convolve_batch(jobs, hcat, scat, yc, precision=prec, seed=77)
            ism.convolve_batch(jobs_n, hcat, scat, yn, precision=prec, seed=77)
            torch.cuda.synchronize()
            yc = yc.cpu().numpy().astype(np.float64)
            yn = yn.cpu().numpy().astype(np.float64)
            o = 0
            for k, (x, s) in enumerate(zip(hs, ss)):
                T = len(s) + x.shape[1] - 1
                c_ = yc[o:o + x.shape[0] * T].reshape(x.shape[0], T)
                g = yn[o:o + x.shape[0] * T].reshape(x.shape[0], T)
                for m in range(x.shape[0]):
                    assert rel_l2(c_[m], refc[k][m]) <= tol, (b, prec, k, m)
                if np.isnan(snr[k]):
                    np.testing.assert_array_equal(g, c_)
                else:
                    ref_n, sigma = oracle.add_noise(c_.copy(), float(snr[k]), 77, ids[k])
                    z = (ref_n - c_) / sigma if sigma > 0 else 0 * c_
                    bar = 2e-6 * sigma * (1 + np.abs(z)) + 2.0 ** -22 * np.abs(c_)
                    assert np.all(np.abs(g - ref_n) <= bar), (b, prec, k)
                o += x.shape[0] * T


def test_random_batches_served_and_host_buffers_bitwise(ism):
    """The same random rooms (RIRs up to 12000 samples) with random sources,
    SNRs (NaN: none) and precision through the host-buffer dataset step at a
    random chunking, and one by one through a server of random batch size
    and stream count: every output equals the batch entry points' bit for
    bit (the dataset step against the batch call, a served request against
    the entry points at the server's 1024-sample window)."""
    import torch
    rng = np.random.default_rng(4)
    done = 0
    while done < 100:
        rooms = [r for r in draw_rooms(rng) if r["rir_len"] <= 12000]
        if not rooms:
            continue
        done += 1
        srcs = [rng.standard_normal(int(rng.integers(1, 6000))).astype(np.float32) for _ in rooms]
        snr = rng.uniform(-5, 40, len(rooms)).astype(np.float32)
        snr[rng.random(len(rooms)) < 0.3] = np.nan
        prec = int(rng.integers(0, 2))
        seed = int(rng.integers(0, 1 << 30))
        lens = [len(s) for s in srcs]
        src_cat = np.concatenate(srcs)
        h = ism.rir_batch(rooms)
        jobs, ylen = ism.conv_jobs([len(r["mics"]) for r in rooms], [r["rir_len"] for r in rooms],
                                   lens, snr_db=snr, noise_ids=np.arange(len(rooms)) + 100)
        y = torch.empty(ylen, device="cuda")
        ism.convolve_batch(jobs, h, torch.from_numpy(src_cat).cuda(), y, seed=seed, precision=prec)
        torch.cuda.synchronize()
        y_ref, h_ref = y.cpu(), h.cpu()
        chunk = int(rng.choice([0, 1, 2, len(rooms)]))
        y_host = torch.full((ylen,), float("nan")).pin_memory()
        h_host = torch.full((h_ref.numel(),), float("nan")).pin_memory()
        ism.dataset_batch(rooms, torch.from_numpy(src_cat).pin_memory(), lens, y_host,
                          snr_db=snr, seed=seed, noise_id_base=100, precision=prec,
                          h_host=h_host, chunk_rooms=chunk)
        assert torch.equal(y_host, y_ref) and torch.equal(h_host, h_ref), (done, chunk, prec)
        with ism.Server(precision=prec, seed=seed, max_batch=int(rng.integers(1, 9)),
                        n_streams=int(rng.integers(1, 4))) as srv:
            tickets = [srv.submit(r, s, float(sn), 100 + i)
                       for i, (r, s, sn) in enumerate(zip(rooms, srcs, snr))]
            for i, (t, r, s, sn) in enumerate(zip(tickets, rooms, srcs, snr)):
                res = srv.wait(t, 60.0)
                M, L, T = res.n_mics, res.rir_len, res.y_len
                hs = torch.empty(M * L, device="cuda")
                ys = torch.empty(M * T, device="cuda")
                srv.copy(t, hs, ys)
                srv.release(t)
                hd = ism.rir_batch([r], window=1024)
                jd, yl = ism.conv_jobs([M], [L], [len(s)], snr_db=[sn], noise_ids=[100 + i])
                yd = torch.empty(yl, device="cuda")
                ism.convolve_batch(jd, hd, torch.from_numpy(s).cuda(), yd, seed=seed, precision=prec)
                torch.cuda.synchronize()
                assert torch.equal(hs.cpu(), hd.cpu()) and torch.equal(ys.cpu(), yd.cpu()), (done, i)
