"""Benchmark of the image-source RIR + convolution hot path on GB300.

One step = one pass of the whole path over one batch: RIRs of 1024 shoebox
rooms (8-mic array, lattice order 15, 81-tap Hann-windowed-sinc fractional
delays, 8192 samples at 16 kHz), then the convolution of each room's 1 s
white-Gaussian source with its 8 RIRs, then Gaussian noise at a per-room SNR
drawn from U[0, 30] dB.  Inputs are synthetic (the paper's recordings are not
available); shapes follow the paper's dataset generation (arXiv 2104.13347,
Sec. II.A, III.A).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("image-source taps/s and mic-samples/s at ≤1e-5 rel-L2; "
          "served p50/p99 latency")
N_ROOMS, N_MICS, ORDER, LH, FS, TS = 1024, 8, 15, 8192, 16000.0, 16000
WORKLOAD = (f"{N_ROOMS} rooms U[3,10]x[3,8]x[2.5,4] m, beta U[0.5,0.95], {N_MICS}-mic 5 cm "
            f"circle, order {ORDER}, 81-tap Hann sinc, RIR {LH} @ 16 kHz; 1 s sources, "
            "SNR U[0,30] dB")


# K1 DRAM traffic per room from the ncu capture summarised in
# profiles/k_ism_sparse_and_k_conv_tcp_1024rooms.md (None when that capture
# predates the current kernel), and the binding resources it measured.
K1_TRAFFIC_PER_ROOM = (33.706752e6 + 15.508480e6) / 256
K1_TRAFFIC_NOTE = ("dram read+write of a 256-room ncu capture, scaled by rooms; reads are "
                   "mostly the per-RIR sorted column lists (15 KB per RIR at order 15), h "
                   "mostly leaves L2 after the kernel, so this understates its 268 MB write")
K1_BINDING = {"issue_active_pct": 78.0, "smem_wavefronts_pct_of_peak": 80.9,
              "fma_pipe_pct": 35.3, "alu_pipe_pct": 42.8, "xu_pipe_pct": 48.9,
              "fp64_pipe_pct": 3.1, "shared_atomic_wavefronts_per_instruction": 3.64,
              "source": "ncu --set full, 256-room case"}
K2_TRAFFIC_PER_ROOM = (83.657984e6 + 138.841088e6) / 256


def k2_live_chunks(ts, lh, kc=64, nn=256, phases=16):
    """Full-width chunk equivalents the persistent tensor-core kernel executes
    for one mic group: its live 64-tap chunks over the time tiles (phases x nn
    outputs), each weighted by the columns its MMAs cover (where the source's
    edge cuts a chunk, only the live columns, in steps of 32; the first chunk
    of a tile at full width)."""
    n_chunks = (lh + phases - 1 + kc - 1) // kc
    n_tiles = -(-(ts + lh - 1) // (phases * nn))
    tot = 0.0
    for t in range(n_tiles):
        c0 = t * phases * nn - lh + 1
        lo = -c0 - (kc - 1 + phases * (nn - 1))
        lo = 0 if lo <= 0 else (lo + kc - 1) // kc
        hi = ts - 1 - c0
        hi = -1 if hi < 0 else hi // kc
        hi = min(hi, n_chunks - 1)
        for i, ch in enumerate(range(lo, hi + 1)):
            width = nn
            if i > 0:
                base = c0 + kc * ch
                nl = max(-((63 + base) >> 4), 0)
                nh = min((ts - 1 - base) >> 4, nn - 1)
                if nl <= nh:
                    width = ((nh | 31) + 1) - (nl & ~31)
            tot += width / nn
    return tot


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9 and p[1].replace(".", "").isdigit():
                        rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    return ws, rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """Largest value over ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank):
    """Each rank generates its own batch of rooms (weak scaling: the units
    are independent rooms, so ranks share no data and exchange nothing)."""
    return 1002 + 7919 * rank


def cpu_sample(rooms, srcs, n_rir_rooms=6, n_conv_rooms=1, single_core=True):
    """Times the oracle (as it stands) on a bounded sample of the workload:
    the RIRs of n_rir_rooms rooms and the convolutions of n_conv_rooms rooms.
    Returns step-equivalent taps/s for the sampled rooms (and, with
    single_core, the same for one room on one core, timed separately)."""
    import oracle
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    hs, st = oracle.rir_batch(rooms[:n_rir_rooms], n_threads=threads)
    t_rir = time.perf_counter() - t0
    t0 = time.perf_counter()
    ys = oracle.convolve_batch(hs[:n_conv_rooms], [s.astype(np.float64) for s in srcs[:n_conv_rooms]],
                               n_threads=threads)
    t_conv = (time.perf_counter() - t0) * n_rir_rooms / n_conv_rooms
    taps = int(st[:, 2].sum())
    mic_samples = n_rir_rooms * N_MICS * (TS + LH - 1)
    single = None
    if single_core:  # one room's RIRs and convolutions on one core
        t0 = time.perf_counter()
        h1, st1 = oracle.rir_batch(rooms[:1], n_threads=1)
        oracle.convolve_batch(h1, [srcs[0].astype(np.float64)], n_threads=1)
        single = int(st1[:, 2].sum()) / (time.perf_counter() - t0)
    return {"value": taps / (t_rir + t_conv), "unit": "taps/s", "cores": threads,
            "kind": "oracle", "single_core_value": single,
            "sample": (f"RIRs of {n_rir_rooms} rooms x {N_MICS} mics of the workload "
                       f"({t_rir:.1f} s) + convolutions of {n_conv_rooms} room(s) scaled to "
                       f"{n_rir_rooms} ({t_conv:.1f} s)"),
            "mic_samples_per_s": mic_samples / (t_rir + t_conv),
            "seconds": t_rir + t_conv, "rirs": hs, "signals": ys}


def parity_vs_sample(ism, cb, h, rooms, srcs, precision):
    """rel-L2 (per room and mic) of the step's RIRs and of a noise-free
    convolution against the oracle outputs of the CPU-baseline sample."""
    import torch
    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    hh = h.view(-1, N_MICS, LH)
    e_h = [rel(hh[i, m].cpu().numpy().astype(np.float64), cb["rirs"][i][m])
           for i in range(len(cb["rirs"])) for m in range(N_MICS)]
    n_c = len(cb["signals"])
    jobs, ylen = ism.conv_jobs([N_MICS] * n_c, [LH] * n_c, [len(x) for x in srcs[:n_c]])
    yc = torch.empty(ylen, device=h.device)
    ism.convolve_batch(jobs, h, torch.from_numpy(np.concatenate(srcs[:n_c])).to(h.device), yc,
                       precision=precision)
    yv = yc.view(n_c, N_MICS, -1).cpu().numpy().astype(np.float64)
    e_y = [rel(yv[i, m], cb["signals"][i][m]) for i in range(n_c) for m in range(N_MICS)]
    return {"rir_rel_l2_max": max(e_h), "rir_rel_l2_median": float(np.median(e_h)),
            "rirs_compared": len(e_h), "signal_rel_l2_max": max(e_y),
            "signal_rel_l2_median": float(np.median(e_y)), "signals_compared": len(e_y),
            "bar": 1e-5, "source": "the oracle outputs of the cpu_baseline sample (noise-free)"}


def run_single_room(ism, wl, dev, stream, reps=200):
    """The single-room case (5 x 4 x 3 m, beta 0.8, order 10, 81 taps, RIR
    4096 @ 16 kHz, one source and one mic): latency per call, device and
    wall clock, for the sparse and direct paths and the allocation-free
    entry point."""
    import torch
    rooms = wl.single_room(seed=1001)
    prep = ism.PreparedRooms(rooms)
    h = torch.empty(prep.h_len, device=dev)
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    ism.rir_batch(rooms, h=h, stats=stats)
    taps = int(stats[1].item())
    contrib = int(stats[0].item())
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {"workload": "5x4x3 m, beta 0.8, order 10 (74088 images), 81 taps, RIR 4096 @ 16 kHz, "
                       "1 source, 1 mic", "taps": taps}
    plan = ism.Plan(prep, h)  # automatic window, as the sparse eager call
    for name, fn in (("sparse", lambda: ism.rir_batch(prep, h=h)),
                     ("sparse_graph", lambda: plan.run(prep)),
                     ("direct", lambda: ism.rir_batch(prep, h=h, variant=ism.RIR_DIRECT)),
                     ("noalloc", lambda: ism.rir_batch_noalloc(rooms, h))):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e[0].record(stream)
        for _ in range(reps):
            fn()
        e[1].record(stream)
        torch.cuda.synchronize()
        out[name] = {"device_us": 1e3 * e[0].elapsed_time(e[1]) / reps,
                     "wall_us": 1e6 * (time.perf_counter() - t0) / reps}
        # one call alone: host work + device time until the result is ready
        lat = []
        for _ in range(20):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            lat.append(1e6 * (time.perf_counter() - t1))
        out[name]["isolated_call_us"] = float(np.median(lat))
    plan.close()
    out["sparse_graph"]["note"] = ("ism_plan_run: the same kernels replayed from a CUDA graph "
                                   "with the room's descriptors copied in")
    # FP32-pipe fraction of the sparse call, on the same algorithmic count as
    # the batch roofline (FIR per output, delay split and terms per image)
    P = ism.rir_filter_terms(0, 81)
    flops = 2.0 * P * 81 * prep.h_len + (40.0 + 2 * P - 1) * contrib
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = 2.0 * 128 * n_sm * peaks()[0].get("sm_max_mhz", 2070.0) * 1e6
    out["sparse"]["fp32_pipe_frac"] = flops / (out["sparse"]["device_us"] * 1e-6) / peak
    out["contributing_images"] = contrib
    return out


def run_plain_path(ism, prep, h, jobs, src, y, stream, ms_step, taps):
    """The same step on the plain GPU path: one RIR launch per room and the
    FP32 direct convolution (same noise, same accuracy bar)."""
    import torch
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ism.rir_batch(prep, h=h, per_room=True)
    ism.convolve_batch(jobs, h, src, y, seed=12345, precision=ism.F32)
    torch.cuda.synchronize()
    e[0].record(stream)
    ism.rir_batch(prep, h=h, per_room=True)
    e[1].record(stream)
    ism.convolve_batch(jobs, h, src, y, seed=12345, precision=ism.F32)
    e[2].record(stream)
    torch.cuda.synchronize()
    rir_ms, conv_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    return {"rir_per_room_ms": rir_ms, "conv_f32_noise_ms": conv_ms, "ms_per_step": rir_ms + conv_ms,
            "value": taps / ((rir_ms + conv_ms) * 1e-3), "unit": "taps/s",
            "speedup_of_the_step": (rir_ms + conv_ms) / ms_step}


def run_ragged(ism, wl, n_requests, dev, stream, n_cmp=128, seconds=1.0):
    """The ragged batch (RT60 U[0.1, 1.0] s, fs 16/48 kHz, 4-16 mics, Sabine
    walls, order from the length): RIRs as one launch at the autotuned
    window; the whole step (RIRs, convolution of a `seconds`-long white
    source per request, noise) eagerly and replayed from a CUDA graph
    (ism_plan_run); the convolution alone (mic-samples/s); and the first
    n_cmp requests' RIRs batched and one launch per room (the plain path)."""
    import torch
    rooms = wl.ragged_batch(n_requests, seed=1005)
    prep = ism.PreparedRooms(rooms)
    n_rirs, hl = ism.rir_batch_size(rooms)
    h = torch.empty(hl, device=dev)
    stats = torch.zeros(2 * n_rirs, dtype=torch.int64, device=dev)
    ism.rir_batch(rooms, h=h, stats=stats, window=ism.WINDOW_TUNE)  # tunes the bucket
    W = ism.rir_tuned_window(prep)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(reps):
            fn()
        e[1].record(stream)
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1]) / reps

    ms = timed(lambda: ism.rir_batch(prep, h=h, window=ism.WINDOW_TUNE), 2)
    ms_auto = timed(lambda: ism.rir_batch(prep, h=h), 2)
    taps = int(stats.view(-1, 2)[:, 1].sum().item())
    # the whole step: sources, convolution (split BF16), noise
    srcs = wl.sources(rooms, seconds, seed=1008)
    lens = [len(x) for x in srcs]
    mics = [len(r["mics"]) for r in rooms]
    src = torch.from_numpy(np.concatenate(srcs)).to(dev)
    snr = wl.snrs(n_requests, seed=1009)
    jobs, ylen = ism.conv_jobs(mics, [r["rir_len"] for r in rooms], lens, snr_db=snr)
    y = torch.empty(ylen, device=dev)
    mic_samples = int(sum(M * (T + r["rir_len"] - 1) for M, T, r in zip(mics, lens, rooms)))

    def eager():
        ism.rir_batch(prep, h=h, window=W)
        ism.convolve_batch(jobs, h, src, y, seed=7, precision=ism.BF16X3)

    ms_conv = timed(lambda: ism.convolve_batch(jobs, h, src, y, seed=7, precision=ism.BF16X3), 2)
    ms_eager = timed(eager, 2)
    y_eager = y.clone()
    plan = ism.Plan(prep, h, src, y, src_lens=lens, precision=ism.BF16X3, window=W, seed=7)
    ms_graph = timed(lambda: plan.run(prep, snr_db=snr), 2)
    same = bool(torch.equal(y, y_eager))
    plan.close()
    del y_eager, y, src
    sub = ism.PreparedRooms(rooms[:n_cmp])
    hs = torch.empty(sub.h_len, device=dev)
    ms_b = timed(lambda: ism.rir_batch(sub, h=hs), 3)
    ms_r = timed(lambda: ism.rir_batch(sub, h=hs, per_room=True), 1)
    del h, hs
    return {"requests": n_requests, "rirs": n_rirs, "samples": hl, "ms": ms,
            "window": W, "window_rule": "autotuned", "ms_automatic_window": ms_auto,
            "taps_per_s": taps / (ms * 1e-3), "rirs_per_s": n_rirs / (ms * 1e-3),
            "workload": "RT60 U[0.1,1.0] s (Sabine walls), fs 16/48 kHz, 4-16 mics, RIR "
                        "ceil(RT60 fs), order from the length, 81-tap Hann sinc; "
                        f"{seconds:g} s white sources, SNR U[0,30] dB",
            "step": {"mic_samples": mic_samples, "conv_ms": ms_conv,
                     "mic_samples_per_s_convolution": mic_samples / (ms_conv * 1e-3),
                     "eager_ms": ms_eager, "graph_ms": ms_graph,
                     "mic_samples_per_s": mic_samples / (ms_graph * 1e-3),
                     "graph_output_bitwise_equal_to_eager": same,
                     "graph": "ism_plan_run: RIRs + split-BF16 convolution + noise of the batch "
                              "replayed from a CUDA graph"},
            "first_requests_batched_vs_per_room": {"requests": n_cmp, "batched_ms": ms_b,
                                                   "per_room_ms": ms_r,
                                                   "speedup": ms_r / ms_b}}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_2104_13347_gb300 import workloads as wl
    rooms = wl.room_batch(N_ROOMS, seed=1002)
    srcs = wl.sources(rooms[:8], 1.0, seed=1003)
    times, last = [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        last = cpu_sample(rooms, srcs, n_rir_rooms=1, n_conv_rooms=1, single_core=False)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    line = {"metric": METRIC, "value": last["value"], "unit": "taps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * statistics.median(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "rooms_per_step": 1,
                       "note": "FP64 CPU oracle, one room's RIRs and convolutions per step"},
            "cpu_baseline": {k: last[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": last["value"], "unit": "taps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_served(ism, wl, rate, seconds, precision, seed=1006, n_streams=16):
    """Serving stream: Poisson arrivals at `rate` req/s for `seconds`; rooms
    U[3,20] m per side, 4-32 mics, fs 16/48 kHz, RT60 U[0.1,0.6] s, sources
    0.5-4 s.  Requests are submitted at their arrival times while earlier
    ones run; latency = submit -> result ready on the device (server clock)."""
    import threading
    n = max(1, int(rate * seconds))
    arrivals, rooms, srcs, snrs = wl.serve_stream(n, rate_hz=rate, seed=seed)
    lat, tickets, rejected = [], [], [0]
    done = threading.Event()
    with ism.Server(precision=precision, seed=seed, max_batch=64, n_streams=n_streams,
                    max_hbm_bytes=32 << 30, max_queue=1 << 16) as srv:
        # warm the kernels and tables outside the measurement
        for i in range(4):
            srv.wait(srv.submit(rooms[i], srcs[i], float(snrs[i])), 120.0)
        # requests marshalled before their arrival times (client-side work;
        # the server copies each source when it is submitted)
        reqs = [srv.request(rooms[i], srcs[i], float(snrs[i])) for i in range(n)]
        q = []
        cv = threading.Condition()

        def waiter():
            k = 0
            while k < n:
                with cv:
                    while len(q) <= k:
                        cv.wait()
                    t = q[k]
                res = srv.wait(t, 600.0)
                lat.append(res.latency_s)
                srv.release(t)
                k += 1
            done.set()

        th = threading.Thread(target=waiter, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for i in range(n):
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            while True:
                try:
                    t = srv.submit(reqs[i])
                    break
                except ism.IsmError as e:  # queue or memory full: retry shortly
                    if e.status != 4:
                        raise
                    rejected[0] += 1
                    time.sleep(0.001)
            with cv:
                q.append(t)
                cv.notify()
        done.wait(600.0)
        wall = time.perf_counter() - t0
        st = srv.stats()
    lat_ms = np.sort(np.asarray(lat)) * 1e3
    return {"rate_req_s": rate, "requests": n, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "completed_req_s": n / wall,
            "taps_per_s": st["taps"] / wall, "mic_samples_per_s": st["mic_samples"] / wall,
            "batches": st["batches"], "busy_retries": rejected[0], "streams": n_streams,
            "host_launch_us_per_batch": st["launch_host_ns"] / 1e3 / max(st["batches"], 1),
            "device_us_per_batch": st["batch_device_ns"] / 1e3 / max(st["batches"], 1),
            "hbm_peak_bytes": st.get("bytes_peak"), "hbm_limit_bytes": 32 << 30,
            "workload": "Poisson arrivals; rooms U[3,20]^3 m, 4-32 mics, fs 16/48 kHz, "
                        "RT60 U[0.1,0.6] s (Sabine), sources 0.5-4 s, SNR U[0,30] dB"}


def run_frames(ism, n_frames, y, n_rooms, T, stream, hbm_gbs, pk_kind):
    """Training frames (1024 samples x 8 mics) cut from the step's convolved
    signals at random rooms and offsets, SNR 20 dB + Exp(10 dB); HBM roofline
    on the frame's read and write."""
    import torch
    rng = np.random.default_rng(31)
    rr = rng.integers(0, n_rooms, n_frames)
    t0 = rng.integers(0, T - 1024, n_frames)
    snr = 20.0 + rng.exponential(10.0, n_frames)
    jobs, n_out = ism.frame_jobs(rr * N_MICS * T, [T] * n_frames, [N_MICS] * n_frames, t0, 1024,
                                 snr_db=snr)
    out = torch.empty(n_out, device=y.device)
    ism.frames_batch(jobs, 1024, y, out, seed=7)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(3):
        ism.frames_batch(jobs, 1024, y, out, seed=7)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / 3
    gbs = 2.0 * n_out * 4 / (ms * 1e-3) / 1e9
    return {"frames": n_frames, "shape": "8 mics x 1024 samples", "ms": ms,
            "frames_per_s": n_frames / (ms * 1e-3),
            "roofline": {"bound": "hbm", "kernel": "k_frames", "achieved": gbs, "peak": hbm_gbs,
                         "unit": "GB/s", "frac": gbs / hbm_gbs,
                         "work": "read + write of every frame sample (8 B)",
                         "peak_note": f"{pk_kind} copy bandwidth"}}


def run_paper_dataset(ism, wl, n_sources, dev, stream):
    """RIR throughput on the paper's own dataset geometry: the 7 x 10 x 3.7 m
    classroom at RT 0.5 s, UMA-8 array, torus sources, 44.1 kHz, delay-limited
    image sets; the 81-tap Hann sinc of the main workload and the paper's
    8-tap Lagrange filter.  Projects the time of one room's 336000 RIRs."""
    import torch
    out = {"workload": f"{n_sources} torus sources x 7 mics, room 7x10x3.7 m, RT 0.5 s "
                       "(Sabine), 44.1 kHz, RIR 22050, order auto"}
    for name, kind, taps in (("hann81", 0, 81), ("lagrange8", 1, 8)):
        rooms = wl.paper_dataset(n_sources, room=1, seed=2021, fd_kind=kind, n_taps=taps)
        n_rirs, hl = ism.rir_batch_size(rooms)
        h = torch.empty(hl, device=dev)
        stats = torch.zeros(2 * n_rirs, dtype=torch.int64, device=dev)
        ism.rir_batch(rooms, h=h, stats=stats)
        prep = ism.PreparedRooms(rooms)
        ism.rir_batch(prep, h=h)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(3):
            ism.rir_batch(prep, h=h)
        e[1].record(stream)
        torch.cuda.synchronize()
        ms = e[0].elapsed_time(e[1]) / 3
        # the same batch at the autotuned window (tuned on its first call)
        ism.rir_batch(prep, h=h, window=ism.WINDOW_TUNE)
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(3):
            ism.rir_batch(prep, h=h, window=ism.WINDOW_TUNE)
        e[1].record(stream)
        torch.cuda.synchronize()
        ms_t = e[0].elapsed_time(e[1]) / 3
        st = stats.view(-1, 2)
        out[name] = {"ms": ms, "rirs": n_rirs, "rirs_per_s": n_rirs / (ms * 1e-3),
                     "window_automatic": 1024, "tuned_window": ism.rir_tuned_window(prep),
                     "tuned_ms": ms_t, "s_per_336000_rirs_tuned": 336000 / (n_rirs / (ms_t * 1e-3)),
                     "taps_per_s": int(st[:, 1].sum().item()) / (ms * 1e-3),
                     "contributing_images_per_rir": int(st[:, 0].sum().item()) / n_rirs,
                     "s_per_336000_rirs": 336000 / (n_rirs / (ms * 1e-3))}
        del h, stats
    return out


def run_ours(args, ws, rank):
    import torch
    import paper_2104_13347_gb300 as ism
    from paper_2104_13347_gb300 import workloads as wl

    ism.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = rank_seed(rank)
    n_rooms = args.rooms
    rooms = wl.room_batch(n_rooms, seed=seed)
    srcs = wl.sources(rooms, 1.0, seed=seed + 1)
    snr = wl.snrs(n_rooms, seed=seed + 2)
    n_rirs, hl = ism.rir_batch_size(rooms)
    jobs, ylen = ism.conv_jobs([N_MICS] * n_rooms, [LH] * n_rooms, [TS] * n_rooms, snr_db=snr,
                               noise_ids=np.arange(n_rooms) + rank * n_rooms)
    precision = ism.BF16X3 if args.precision == "bf16x3" else ism.F32
    stream = torch.cuda.current_stream()
    src_host = torch.from_numpy(np.concatenate(srcs)).pin_memory()
    src = src_host.to(dev)
    h = torch.empty(hl, device=dev)
    y = torch.empty(ylen, device=dev)
    stats = torch.zeros(2 * n_rirs, dtype=torch.int64, device=dev)
    prep = ism.PreparedRooms(rooms)  # rooms marshalled once, outside the timed region

    variant = ism.RIR_DIRECT if args.rir_variant == "direct" else ism.RIR_SPARSE
    ism.rir_batch(rooms, h=h, stats=stats, window=args.window, variant=variant)
    torch.cuda.synchronize()
    taps = int(stats.view(-1, 2)[:, 1].sum().item())
    mic_samples = n_rooms * N_MICS * (TS + LH - 1)

    # per-step stage events, read after the timed region (no host sync inside)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        ism.rir_batch(prep, h=h, window=args.window, variant=variant)
        if ev:
            ev[1].record(stream)
        ism.convolve_batch(jobs, h, src, y, seed=12345, precision=precision)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clocks:
        start.record(stream)
        for i in range(args.steps):
            step(evs[i])
        end.record(stream)
        torch.cuda.synchronize()
    rir_ms = [e[0].elapsed_time(e[1]) for e in evs]
    conv_ms = [e[1].elapsed_time(e[2]) for e in evs]
    barrier(ws)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(start.elapsed_time(end), ws)
    ms_step = total_ms / args.steps
    clk = clocks.summary()

    # end to end through the C-ABI call with HOST buffers (ism_dataset_batch):
    # pinned sources in, noisy microphone signals out, every copy inside the
    # timed region; the call overlaps the copies of one chunk of rooms with
    # the kernels of another and returns when y is in host memory
    y_host = torch.empty(ylen, dtype=torch.float32).pin_memory()
    lens = [TS] * n_rooms
    e2e_steps = max(1, min(args.steps, 5))
    ism.dataset_batch(prep, src_host, lens, y_host, snr_db=snr, seed=12345,
                      noise_id_base=rank * n_rooms, precision=precision)
    barrier(ws)
    t_e = time.perf_counter()
    for _ in range(e2e_steps):
        ism.dataset_batch(prep, src_host, lens, y_host, snr_db=snr, seed=12345,
                          noise_id_base=rank * n_rooms, precision=precision)
    e2e_ms = max_over_ranks((time.perf_counter() - t_e) * 1e3, ws) / e2e_steps
    # the same step with the copies and kernels in sequence on one stream
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e_start.record(stream)
    for _ in range(e2e_steps):
        src.copy_(src_host, non_blocking=True)
        ism.rir_batch(prep, h=h, window=args.window, variant=variant)
        ism.convolve_batch(jobs, h, src, y, seed=12345, precision=precision)
        y_host.copy_(y, non_blocking=True)
    e_end.record(stream)
    torch.cuda.synchronize()
    e2e_serial_ms = max_over_ranks(e_start.elapsed_time(e_end), ws) / e2e_steps

    pk, pk_kind = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    rir_med = statistics.median(rir_ms)
    conv_med = statistics.median(conv_ms)
    contrib = int(stats.view(-1, 2)[:, 0].sum().item())
    P = ism.rir_filter_terms(0, 81)
    # K1 (sparse path) algorithmic FP32 work per launch: per contributing
    # image 40 flops for the float-float delay split and the gain, and 2P - 1
    # for the P Chebyshev terms (recurrence on the scaled gain); per output
    # sample 2 P n_taps for the FIR.  Peak: FP32 FMA pipe, 128 lanes x 2
    # flops per clock per SM at the maximum SM clock.
    k1_flops = 2.0 * P * 81 * n_rirs * LH + (40.0 + 2 * P - 1) * contrib
    peak_fp32 = 2.0 * 128 * n_sm * sm_mhz * 1e6
    k1_rate = k1_flops / (rir_med * 1e-3)
    # context: the direct per-tap formulation is bound by the reciprocal
    # (MUFU) pipe, 16 results per clock per SM, one per tap
    direct_bound = 16.0 * n_sm * sm_mhz * 1e6
    # context: the sparse path's binding resource is the shared-memory pipe,
    # two thirds of it the P u32 atomics per contributing image; 32 lanes at
    # random addresses complete 9.1 atomics per clock per SM on this GPU
    # (a loop of random-address u32 shared atomics, 3.5 wavefronts each)
    atom_rate = P * contrib / (rir_med * 1e-3)
    atom_peak = 9.1 * n_sm * sm_mhz * 1e6

    # K2 alone (no noise), timed back to back: split-BF16 needs at least the
    # three products hi.hi, hi.lo, lo.hi of 2 Ts Lh flops per mic; the kernel
    # executes those three, as 12 MMAs of 128 x N x 16 per live 64-tap chunk
    # of a 4096-output tile (N = 256, or the live columns where the source's
    # edge cuts the chunk; the padding at the tile edges is the rest)
    jobs_clean, _ = ism.conv_jobs([N_MICS] * n_rooms, [LH] * n_rooms, [TS] * n_rooms)
    k2_ms = None
    if precision == ism.BF16X3:
        k2e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ism.convolve_batch(jobs_clean, h, src, y, precision=precision)
        k2e[0].record(stream)
        for _ in range(3):
            ism.convolve_batch(jobs_clean, h, src, y, precision=precision)
        k2e[1].record(stream)
        torch.cuda.synchronize()
        k2_ms = k2e[0].elapsed_time(k2e[1]) / 3
    k2_alg = 3 * 2.0 * TS * LH * n_rooms * N_MICS
    k2_exec = 12 * 2.0 * 128 * 256 * 16 * k2_live_chunks(TS, LH) * n_rooms
    bf16_peak = pk.get("bf16_tflops", 1900.0) * 1e12
    line = {
        "metric": METRIC, "value": ws * taps / (ms_step * 1e-3), "unit": "taps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if precision == ism.F32 else "bf16x3+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if n_rooms == N_ROOMS else
                   WORKLOAD.replace(f"{N_ROOMS} rooms", f"{n_rooms} rooms"), "rooms": n_rooms, "mics": N_MICS, "order": ORDER,
                   "rir_len": LH, "src_len": TS, "n_taps": 81,
                   "window": (ism.rir_tuned_window(prep, variant) if args.window < 0 else
                              args.window or 1024),
                   "window_rule": {-1: "autotuned", 0: "automatic"}.get(args.window, "fixed"),
                   "precision": args.precision, "parallelism": f"replicas x{ws}",
                   "l2": f"inputs larger than L2 (h {hl * 4 / 1e6:.0f} MB, y {ylen * 4 / 1e6:.0f} MB "
                         "per step), no flush"},
        "secondary": {"mic_samples_per_s": ws * mic_samples / (ms_step * 1e-3),
                      "mic_samples_per_s_convolution": ws * mic_samples / (conv_med * 1e-3),
                      "taps_per_step": taps, "mic_samples_per_step": mic_samples,
                      "stage_ms": {"rir": rir_med, "conv_noise": conv_med}},
        "roofline": {"bound": "alu", "kernel": "k_ism_sparse" if args.rir_variant == "sparse" else "k_ism_taps", "achieved": k1_rate / 1e12,
                     "peak": peak_fp32 / 1e12, "unit": "TFLOP/s", "frac": k1_rate / peak_fp32,
                     "traffic": K1_TRAFFIC_PER_ROOM * n_rooms if K1_TRAFFIC_PER_ROOM else None,
                     "traffic_note": K1_TRAFFIC_NOTE,
                     "work": f"2*P*n_taps per output (FIR) + 40+2P-1 per contributing image, P={P}",
                     "peak_note": f"FP32 FMA pipe, 128 lanes x 2 flop/clk/SM x {n_sm} SMs x "
                                  f"{sm_mhz:.0f} MHz ({pk_kind} max clock)",
                     "binding": K1_BINDING,
                     "taps_per_s": taps / (rir_med * 1e-3),
                     "direct_formulation_bound_taps_per_s": direct_bound,
                     "k1_ms": rir_med,
                     # the binding resource of K1: shared-memory atomics
                     "shared_atomics_per_s": atom_rate, "shared_atomics_peak_per_s": atom_peak,
                     "shared_atomics_frac": atom_rate / atom_peak,
                     # K2 (tensor-core convolution, timed alone), scalars so
                     # that every reader of the line keeps them
                     "k2_kernel": "k_conv_tcp",
                     "k2_ms": k2_ms,
                     "k2_achieved_tflops": None if k2_ms is None else k2_alg / (k2_ms * 1e-3) / 1e12,
                     "k2_peak_tflops": bf16_peak / 1e12,
                     "k2_frac": None if k2_ms is None else k2_alg / (k2_ms * 1e-3) / bf16_peak,
                     "k2_executed_frac": None if k2_ms is None else
                     k2_exec / (k2_ms * 1e-3) / bf16_peak,
                     "k2_traffic": K2_TRAFFIC_PER_ROOM * n_rooms},
        "roofline_k2": None if k2_ms is None else {
            "bound": "tensor", "kernel": "k_conv_tcp", "achieved": k2_alg / (k2_ms * 1e-3) / 1e12,
            "peak": bf16_peak / 1e12, "unit": "TFLOP/s",
            "frac": k2_alg / (k2_ms * 1e-3) / bf16_peak,
            "executed_tflops": k2_exec / (k2_ms * 1e-3) / 1e12,
            "executed_frac": k2_exec / (k2_ms * 1e-3) / bf16_peak, "ms": k2_ms,
            "traffic": K2_TRAFFIC_PER_ROOM * n_rooms,
            "traffic_note": "dram read+write of a 256-room ncu capture, scaled by rooms",
            "work": "3 x 2 Ts Lh per mic (split-BF16 minimum); executed: 12 MMAs 128xNx16 "
                    "per live 64-tap chunk per 4096-output tile (N = 256 or the chunk's live "
                    "columns)",
            "peak_note": f"dense bf16, {pk_kind} burst (kernel timed alone)"},
        "e2e": {"value": ws * taps / (e2e_ms * 1e-3), "unit": "taps/s",
                "h2d_bytes_per_step": int(src_host.numel() * 4),
                "d2h_bytes_per_step": int(ylen * 4), "ms_per_step": e2e_ms,
                "api": "ism_dataset_batch (host buffers, pinned; copies overlap kernels by chunk)",
                "serial_ms_per_step": e2e_serial_ms},
        "gpu_launches": args.steps * 4,  # K1 tables + K1, convolution (noise partials fused), noise
        "clocks": clk,
    }
    if args.frames > 0:
        line["frames"] = run_frames(ism, args.frames, y, n_rooms, TS + LH - 1, stream,
                                    pk.get("hbm_gbs", 6800.0), pk_kind)
    if args.paper_sources > 0:
        line["paper_dataset"] = run_paper_dataset(ism, wl, args.paper_sources, dev, stream)
    line["single_room"] = run_single_room(ism, wl, dev, stream)
    if args.plain_path:
        line["plain_path"] = run_plain_path(ism, prep, h, jobs, src, y, stream, ms_step, taps)
    if args.ragged > 0:
        line["ragged"] = run_ragged(ism, wl, args.ragged, dev, stream)
    rates = [float(r) for r in args.serve_rates.split(",") if r] if args.serve_rate > 0 else []
    if rates:
        line["served"] = [run_served(ism, wl, r, args.serve_seconds, precision,
                                     n_streams=args.serve_streams) for r in rates]
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_sample(rooms, srcs)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                   "single_core_value")}
        line["parity"] = parity_vs_sample(ism, cb, h, rooms, srcs, precision)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["f32", "bf16x3"],
                    help="convolution arithmetic (both meet 1e-5 rel-L2 on this workload)")
    ap.add_argument("--window", type=int, default=-1,
                    help="K1 window: -1 = the library's autotuner (default), 0 = automatic "
                         "rule, or a multiple of 32")
    ap.add_argument("--rir-variant", default="sparse", choices=["sparse", "direct"],
                    help="K1 kernel: sparse Chebyshev arrays (default) or the direct per-tap one")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=1.0,
                    help="0 skips the served streams (their rates: --serve-rates)")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-streams", type=int, default=16,
                    help="streams of the server (batches in flight at once)")
    ap.add_argument("--serve-rates", default="200,1000,5000",
                    help="Poisson rates (req/s) of the served streams, comma-separated")
    ap.add_argument("--plain-path", type=int, default=1,
                    help="1: also time the step on the plain path (per-room RIR launches, "
                         "FP32 convolution)")
    ap.add_argument("--ragged", type=int, default=4096,
                    help="requests of the ragged-batch measurement (0 = skip)")
    ap.add_argument("--frames", type=int, default=65536,
                    help="training frames of the frame measurement (0 = skip)")
    ap.add_argument("--paper-sources", type=int, default=2048,
                    help="sources of the paper-dataset RIR measurement (0 = skip)")
    ap.add_argument("--rooms", type=int, default=N_ROOMS,
                    help="rooms per step (smaller only for profiling captures)")
    args = ap.parse_args()
    ws, rank = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
