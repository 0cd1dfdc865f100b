"""GPU tests of the continuous-batching server (ism_serve_*).

Requests of uneven sizes are submitted while others are on the GPU; each
result must equal the batch entry points' on the same inputs and be the
same alone and in the mix (bit for bit: the RIR sums are fixed-point and a
job's convolution tiles depend on the job alone), and match the FP64 oracle
at the path's bars (arXiv 2104.13347
Sec. II.A RIR + convolution, Sec. III.A noise).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def requests(n, seed):
    """Small mixed requests: 1-9 mics, RIRs 300-5000 samples, sources of
    500-6000 samples, orders 2-6, some with noise."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        room = wl.room_batch(1, seed=seed * 1000 + i, order=int(rng.integers(2, 7)),
                             rir_len=int(rng.integers(300, 5000)),
                             n_mics=int(rng.integers(1, 10)))[0]
        src = rng.standard_normal(int(rng.integers(500, 6000))).astype(np.float32)
        snr = float(rng.uniform(0, 30)) if i % 3 == 0 else math.nan
        out.append((room, src, snr, 7000 + i))
    return out


def fetch(ism, srv, ticket, room, src):
    import torch
    res = srv.wait(ticket, 60.0)
    M, L, T = res.n_mics, res.rir_len, res.y_len
    assert M == len(room["mics"]) and L == room["rir_len"] and T == len(src) + L - 1
    h = torch.empty(M * L, device="cuda")
    y = torch.empty(M * T, device="cuda")
    srv.copy(ticket, h, y)
    torch.cuda.synchronize()
    return (h.cpu().numpy().reshape(M, L).astype(np.float64),
            y.cpu().numpy().reshape(M, T).astype(np.float64), res)


def direct(ism, room, src, snr, noise_id, seed, precision):
    """The same request through the batch entry points (with the server's
    1024-sample RIR windows)."""
    import torch
    h = ism.rir_batch([room], window=1024)
    jobs, ylen = ism.conv_jobs([len(room["mics"])], [room["rir_len"]], [len(src)],
                               snr_db=[snr], noise_ids=[noise_id])
    y = torch.empty(ylen, device="cuda")
    ism.convolve_batch(jobs, h, torch.from_numpy(src).cuda(), y, seed=seed,
                       precision=precision)
    torch.cuda.synchronize()
    M, L = len(room["mics"]), room["rir_len"]
    return (h.cpu().numpy().reshape(M, L).astype(np.float64),
            y.cpu().numpy().reshape(M, -1).astype(np.float64))


@pytest.mark.parametrize("precision", [0, 1])
def test_serve_mix_matches_batch_api_and_alone(ism, precision):
    reqs = requests(24, seed=3)
    seed = 99
    with ism.Server(precision=precision, seed=seed, max_batch=8, n_streams=3) as srv:
        tickets = [srv.submit(r, s, snr, nid) for r, s, snr, nid in reqs]
        mixed = [fetch(ism, srv, t, r, s) for t, (r, s, _, _) in zip(tickets, reqs)]
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["batches"] >= 2
        for t in tickets:
            srv.release(t)
    # alone: a fresh server per request
    for k in (0, 5, 17):
        r, s, snr, nid = reqs[k]
        with ism.Server(precision=precision, seed=seed) as srv:
            t = srv.submit(r, s, snr, nid)
            h1, y1, _ = fetch(ism, srv, t, r, s)
        h0, y0, _ = mixed[k]
        # a request's work items do not depend on the mix: bit for bit
        np.testing.assert_array_equal(h0, h1)
        np.testing.assert_array_equal(y0, y1)
    # batch entry points on the same inputs: the same kernels, whose work for
    # a job does not depend on the rest of the batch -- bit for bit
    for k in (1, 6, 12):
        r, s, snr, nid = reqs[k]
        hd, yd = direct(ism, r, s, snr, nid, seed, precision)
        np.testing.assert_array_equal(mixed[k][0], hd)
        np.testing.assert_array_equal(mixed[k][1], yd)


@pytest.mark.parametrize("precision", [0, 1])
def test_serve_parity_with_oracle(ism, precision):
    """Served RIRs and signals against the FP64 oracle: the FP32 convolution
    and the split-BF16 persistent tensor-core kernel of the batch calls."""
    reqs = requests(4, seed=5)
    with ism.Server(precision=precision) as srv:
        tickets = [srv.submit(r, s) for r, s, _, _ in reqs]  # no noise
        for t, (r, s, _, _) in zip(tickets, reqs):
            h, y, res = fetch(ism, srv, t, r, s)
            href, _ = oracle.rir_batch([r])
            yref = oracle.convolve_batch([href[0]], [s.astype(np.float64)])[0]
            for m in range(h.shape[0]):
                assert rel_l2(h[m], href[0][m]) <= 1e-5
                assert rel_l2(y[m], yref[m]) <= 1e-5
            assert res.latency_s >= res.queue_s >= 0
            srv.release(t)


def test_serve_hbm_admission_queues_requests(ism):
    """A device budget that holds only a couple of requests at a time: all
    requests still complete, the budget is never exceeded."""
    reqs = requests(12, seed=7)
    budget = 3 << 20
    with ism.Server(max_hbm_bytes=budget, max_batch=4, n_streams=2) as srv:
        tickets = [srv.submit(r, s) for r, s, _, _ in reqs]
        for t, (r, s, _, _) in zip(tickets, reqs):
            fetch(ism, srv, t, r, s)
            srv.release(t)  # frees memory so queued requests can be admitted
        st = srv.stats()
        assert st["completed"] == len(reqs)
        assert 0 < st["bytes_peak"] <= budget
        assert st["taps"] > 0 and st["mic_samples"] > 0


def test_serve_split_bf16_short_rirs_against_oracle(ism):
    """Served split-BF16 requests with RIRs from a few hundred samples to
    ~8.7k and partial 8-mic groups, each (request, mic) against the
    oracle's convolution of the served RIR and the served RIR against the
    oracle's RIR (1e-5 rel-L2 each)."""
    rng = np.random.default_rng(41)
    shapes = [(1, 200, 3000), (5, 1000, 700), (8, 2048, 4100), (12, 4097, 2500),
              (3, 8700, 1500), (9, 333, 9000)]
    reqs = []
    for i, (M, L, T) in enumerate(shapes):
        room = wl.room_batch(1, seed=4100 + i, order=int(rng.integers(2, 6)), rir_len=L,
                             n_mics=M)[0]
        reqs.append((room, rng.standard_normal(T).astype(np.float32)))
    with ism.Server(precision=1, max_batch=3, n_streams=2) as srv:
        tickets = [srv.submit(r, s) for r, s in reqs]
        for t, (r, s) in zip(tickets, reqs):
            h, y, _ = fetch(ism, srv, t, r, s)
            href, _ = oracle.rir_batch([r])
            yref = oracle.convolve_batch([h], [s.astype(np.float64)])[0]
            for m in range(h.shape[0]):
                assert rel_l2(h[m], href[0][m]) <= 1e-5, (r["rir_len"], m)
                assert rel_l2(y[m], yref[m]) <= 1e-5, (r["rir_len"], m)
            srv.release(t)


def test_serve_split_bf16_long_rirs_against_oracle(ism):
    """Served split-BF16 requests with long RIRs (30000 and 40000 samples),
    each (request, mic) against the oracle's convolution of the served RIR
    (1e-5 rel-L2: short sources, a few thousand terms per output)."""
    rng = np.random.default_rng(43)
    reqs = []
    for i, (M, L, T) in enumerate([(2, 30000, 3000), (3, 40000, 2500)]):
        room = wl.room_batch(1, seed=4300 + i, order=5, rir_len=L, n_mics=M)[0]
        reqs.append((room, rng.standard_normal(T).astype(np.float32)))
    with ism.Server(precision=1, max_batch=2, n_streams=2) as srv:
        tickets = [srv.submit(r, s) for r, s in reqs]
        for t, (r, s) in zip(tickets, reqs):
            h, y, _ = fetch(ism, srv, t, r, s)
            yref = oracle.convolve_batch([h], [s.astype(np.float64)])[0]
            for m in range(h.shape[0]):
                assert rel_l2(y[m], yref[m]) <= 1e-5, (r["rir_len"], m)
            srv.release(t)


def test_serve_long_source_in_segment_windows(ism):
    """A served split-BF16 request whose tiles need more than one source
    window (RIR 30000 samples, source 26000): its signals equal the batch
    call's on the served RIR bit for bit (the same kernel, a job's tiles do
    not depend on the batch), and the oracle's convolution within the 2e-4
    the specification sets for the split-BF16 convolution (tens of
    thousands of terms per output)."""
    import torch
    rng = np.random.default_rng(47)
    room = wl.room_batch(1, seed=4700, order=5, rir_len=30000, n_mics=3)[0]
    src = rng.standard_normal(26000).astype(np.float32)
    with ism.Server(precision=1) as srv:
        t = srv.submit(room, src)
        h, y, _ = fetch(ism, srv, t, room, src)
        srv.release(t)
    jobs, ylen = ism.conv_jobs([3], [30000], [len(src)])
    yb = torch.empty(ylen, device="cuda")
    ism.convolve_batch(jobs, torch.from_numpy(h.astype(np.float32).ravel()).cuda(),
                       torch.from_numpy(src).cuda(), yb, precision=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y, yb.cpu().numpy().astype(np.float64).reshape(y.shape))
    yref = oracle.convolve_batch([h], [src.astype(np.float64)])[0]
    for m in range(3):
        assert rel_l2(y[m], yref[m]) <= 2e-4, m
