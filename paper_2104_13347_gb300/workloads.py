"""Seeded synthetic inputs shaped like the paper's RIR workloads.

This module only draws inputs (room sizes, wall coefficients, source and
microphone positions, source signals, SNRs, arrival times).  It contains none
of the image-source or convolution arithmetic, imports nothing from the CUDA
binding or from the oracle, and is the one module both sides take inputs
from.

The paper (arXiv 2104.13347, Sec. II.A and III.A) simulates 7 x 10 x 3.7 m
and 5 x 5 x 4 m rooms at RT 0.5 s with a 7-mic compact array and convolves
music, speech and urban recordings; those recordings are not available, so
white Gaussian sources stand in for them, and the room, array and signal
distributions below are the synthetic stand-ins used for measurement.
"""
from __future__ import annotations

import math

import numpy as np

FD_HANN_SINC = 0
FD_LAGRANGE = 1


def _uniform_point(rng, dims, clearance):
    lo = np.full(3, clearance)
    hi = np.asarray(dims, float) - clearance
    return lo + (hi - lo) * rng.random(3)


def circular_array(center, n_mics, radius):
    """Horizontal circle, mic i at angle 2 pi i / M around `center`."""
    ang = 2.0 * np.pi * np.arange(n_mics) / n_mics
    m = np.empty((n_mics, 3))
    m[:, 0] = center[0] + radius * np.cos(ang)
    m[:, 1] = center[1] + radius * np.sin(ang)
    m[:, 2] = center[2]
    return m


def single_room(seed=1001, order=10, rir_len=4096, n_taps=81, fd_kind=FD_HANN_SINC):
    """5 x 4 x 3 m room, all walls beta = 0.8, one source and one mic drawn
    uniformly with 0.5 m wall clearance, fs 16 kHz, c 343 m/s."""
    rng = np.random.default_rng(seed)
    dims = np.array([5.0, 4.0, 3.0])
    src = _uniform_point(rng, dims, 0.5)
    mic = _uniform_point(rng, dims, 0.5)
    return [dict(dims=dims, beta=np.full(6, 0.8), src=src, mics=mic[None, :], fs=16000.0,
                 c=343.0, order=order, n_taps=n_taps, fd_kind=fd_kind, rir_len=rir_len)]


def room_batch(n_rooms=1024, seed=1002, order=15, rir_len=8192, n_mics=8, radius=0.05,
               n_taps=81, fd_kind=FD_HANN_SINC, fs=16000.0):
    """Batch of rooms: dims U[3,10] x U[3,8] x U[2.5,4] m, per-wall beta
    U[0.5, 0.95], one source (0.5 m clearance) and an 8-mic circular array of
    radius 5 cm whose centre keeps 0.5 m + r clearance."""
    rng = np.random.default_rng(seed)
    rooms = []
    for _ in range(n_rooms):
        dims = np.array([rng.uniform(3, 10), rng.uniform(3, 8), rng.uniform(2.5, 4)])
        beta = rng.uniform(0.5, 0.95, 6)
        src = _uniform_point(rng, dims, 0.5)
        ctr = _uniform_point(rng, dims, 0.5 + radius)
        rooms.append(dict(dims=dims, beta=beta, src=src,
                          mics=circular_array(ctr, n_mics, radius), fs=fs, c=343.0,
                          order=order, n_taps=n_taps, fd_kind=fd_kind, rir_len=rir_len))
    return rooms


def sources(rooms, seconds=1.0, seed=1003):
    """White Gaussian float32 source per room (unit variance), `seconds`
    long at the room's sampling rate (a scalar or one value per room)."""
    rng = np.random.default_rng(seed)
    secs = np.broadcast_to(np.asarray(seconds, float), (len(rooms),))
    return [rng.standard_normal(int(round(s * r["fs"]))).astype(np.float32)
            for r, s in zip(rooms, secs)]


def snrs(n, lo=0.0, hi=30.0, seed=1004):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n).astype(np.float32)


def sabine_beta(dims, rt60):
    """Wall reflection coefficient from a target RT60 through Sabine's
    formula alpha = 0.161 V / (S RT60), clamped to [0, 1], beta = sqrt(1-alpha)."""
    L = np.asarray(dims, float)
    V = float(np.prod(L))
    S = 2.0 * (L[0] * L[1] + L[0] * L[2] + L[1] * L[2])
    alpha = min(1.0, max(0.0, 0.161 * V / (S * rt60)))
    return math.sqrt(1.0 - alpha)


def eyring_beta(dims, rt60):
    """Wall reflection coefficient from a target RT60 through Eyring's
    formula RT60 = 0.161 V / (-S ln(1 - alpha)): alpha = 1 - exp(-0.161 V /
    (S RT60)), beta = sqrt(1 - alpha) = exp(-0.0805 V / (S RT60)).  Eyring's
    law is the one a uniform image lattice obeys at first: its images cross
    S / (4V) walls per metre on average, so with these walls the energy of
    the image sum starts to decay at 60 dB per RT60.  Unlike Sabine's alpha
    it never reaches 1, so any RT60 > 0 gives walls in (0, 1)."""
    L = np.asarray(dims, float)
    V = float(np.prod(L))
    S = 2.0 * (L[0] * L[1] + L[0] * L[2] + L[1] * L[2])
    return math.exp(-0.5 * 0.161 * V / (S * rt60))


def wall_beta(dims, rt60, walls="sabine"):
    """beta on all six walls for RT60 by `walls` = "sabine" or "eyring"."""
    if walls == "sabine":
        return sabine_beta(dims, rt60)
    if walls == "eyring":
        return eyring_beta(dims, rt60)
    raise ValueError(f"walls must be 'sabine' or 'eyring', not {walls!r}")


def order_for_length(dims, rir_len, fs, c, n_taps):
    """Smallest lattice order whose images cover every delay up to the RIR
    length plus the filter half-width, on every axis (plus one)."""
    H = (n_taps - 1) // 2
    reach = c * rir_len / fs + (H + 1) * c / fs
    return int(max(math.ceil(reach / (2.0 * L)) for L in dims) + 1)


def ragged_batch(n_requests=4096, seed=1005, rt_lo=0.1, rt_hi=1.0, n_taps=81,
                 max_order=None, walls="sabine"):
    """Ragged requests: RT60 U[rt_lo, rt_hi] s, fs in {16, 48} kHz, RIR length
    ceil(RT60 fs), beta on all six walls from Sabine (or Eyring, `walls`),
    order from the length, 4..16 mics on a 5 cm circle, dims as in
    `room_batch`."""
    rng = np.random.default_rng(seed)
    rooms = []
    for _ in range(n_requests):
        dims = np.array([rng.uniform(3, 10), rng.uniform(3, 8), rng.uniform(2.5, 4)])
        rt60 = rng.uniform(rt_lo, rt_hi)
        fs = 16000.0 if rng.random() < 0.5 else 48000.0
        rir_len = int(math.ceil(rt60 * fs))
        n_mics = int(rng.integers(4, 17))
        src = _uniform_point(rng, dims, 0.5)
        ctr = _uniform_point(rng, dims, 0.55)
        order = order_for_length(dims, rir_len, fs, 343.0, n_taps)
        if max_order is not None:
            order = min(order, max_order)
        rooms.append(dict(dims=dims, beta=np.full(6, wall_beta(dims, rt60, walls)), src=src,
                          mics=circular_array(ctr, n_mics, 0.05), fs=fs, c=343.0,
                          order=order, n_taps=n_taps, fd_kind=FD_HANN_SINC,
                          rir_len=rir_len, rt60=rt60))
    return rooms


def serve_stream(n_requests=256, rate_hz=1000.0, seed=1006, rt_lo=0.1, rt_hi=0.6,
                 src_lo=0.5, src_hi=4.0, mic_lo=4, mic_hi=32, max_order=None, n_taps=81,
                 walls="sabine"):
    """Poisson arrivals at `rate_hz`; rooms U[3,20] m per side; 4..32 mics;
    fs 16/48 kHz; sources 0.5..4 s; RT60 and walls as in `ragged_batch`.
    Returns (arrival times in s, rooms, sources, snrs)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    rooms, srcs = [], []
    for _ in range(n_requests):
        dims = rng.uniform(3, 20, 3)
        rt60 = rng.uniform(rt_lo, rt_hi)
        fs = 16000.0 if rng.random() < 0.5 else 48000.0
        rir_len = int(math.ceil(rt60 * fs))
        n_mics = int(rng.integers(mic_lo, mic_hi + 1))
        order = order_for_length(dims, rir_len, fs, 343.0, n_taps)
        if max_order is not None:
            order = min(order, max_order)
        src = _uniform_point(rng, dims, 0.5)
        ctr = _uniform_point(rng, dims, 0.55)
        rooms.append(dict(dims=dims, beta=np.full(6, wall_beta(dims, rt60, walls)), src=src,
                          mics=circular_array(ctr, n_mics, 0.05), fs=fs, c=343.0,
                          order=order, n_taps=n_taps, fd_kind=FD_HANN_SINC, rir_len=rir_len))
        srcs.append(rng.standard_normal(int(rng.uniform(src_lo, src_hi) * fs)).astype(np.float32))
    return t, rooms, srcs, rng.uniform(0, 30, n_requests).astype(np.float32)


# ---------------------------------------------------------------------------
# The paper's own dataset geometry (Sec. II.A and III.A; the recordings and
# the trained network are not available, so only the geometry is drawn)
# ---------------------------------------------------------------------------

# Room 1: 7 x 10 x 3.7 m classroom with the array at [4, 6, 1.5]; room 2:
# 5 x 5 x 4 m, array position not stated (taken at the horizontal centre,
# 1.5 m high); both at RT 0.5 s.  Frames of 1024 samples last 23.2 ms, so
# fs = 44.1 kHz.
PAPER_ROOMS = {
    1: (np.array([7.0, 10.0, 3.7]), np.array([4.0, 6.0, 1.5])),
    2: (np.array([5.0, 5.0, 4.0]), np.array([2.5, 2.5, 1.5])),
}
PAPER_FS = 44100.0
PAPER_RT = 0.5


def uma8_array(center, radius=0.04):
    """7 microphones: one at the centre and six on a horizontal circle of
    radius 4 cm (8 cm diameter) around it."""
    ring = circular_array(center, 6, radius)
    return np.vstack([np.asarray(center, float)[None, :], ring])


def torus_sources(n, center, dims, seed=1007, R=2.0, dR=0.5, dphi_deg=7.0, clearance=0.1):
    """Source positions in the torus around the array centre: distance
    U[R - dR, R + dR], azimuth U[0, 2 pi), elevation U[-dphi, dphi]; draws
    closer than `clearance` to a wall are redrawn."""
    rng = np.random.default_rng(seed)
    c0 = np.asarray(center, float)
    L = np.asarray(dims, float)
    out = np.empty((n, 3))
    k = 0
    while k < n:
        r = rng.uniform(R - dR, R + dR)
        th = rng.uniform(0.0, 2.0 * np.pi)
        ph = np.deg2rad(rng.uniform(-dphi_deg, dphi_deg))
        p = c0 + r * np.array([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)])
        if np.all(p > clearance) and np.all(p < L - clearance):
            out[k] = p
            k += 1
    return out


def paper_dataset(n_sources=1024, room=1, seed=1007, fd_kind=FD_HANN_SINC, n_taps=81, rt=None,
                  walls="sabine"):
    """One request per source position: the paper room `room` (1 or 2) at
    RT 0.5 s (Sabine walls, or Eyring: `walls`), the UMA-8 array, fs 44.1
    kHz, RIR length RT fs,
    and the delay-limited image set (order -1 = automatic).  fd_kind
    FD_LAGRANGE with n_taps 8 is the paper's own 7th-order filter."""
    dims, ctr = PAPER_ROOMS[room]
    rt = PAPER_RT if rt is None else rt
    mics = uma8_array(ctr)
    beta = np.full(6, wall_beta(dims, rt, walls))
    srcs = torus_sources(n_sources, ctr, dims, seed=seed)
    L = int(round(rt * PAPER_FS))
    return [dict(dims=dims, beta=beta, src=s, mics=mics, fs=PAPER_FS, c=343.0, order=-1,
                 n_taps=n_taps, fd_kind=fd_kind, rir_len=L) for s in srcs]
