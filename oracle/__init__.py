"""FP64 CPU oracle for the image-source RIR and convolution path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path (the CUDA library
and its binding) never imports this package, and this package imports
nothing from the product.

The arithmetic lives in ``ism_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module compiles it on first use and exposes it
through ctypes with numpy arrays.  Every function follows arXiv 2104.13347,
Sec. II.A (image sources, delays, wall dampings, fractional-delay taps, batch
convolution) and Sec. III.A (Gaussian noise at a drawn SNR).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_SRC / ORACLE_BUILD let the mutation test compile a deliberately
# broken copy of the oracle into a scratch folder and check that the pins
# reject it.
_SRC = os.environ.get("ORACLE_SRC", os.path.join(_HERE, "ism_oracle.c"))
_BUILD = os.environ.get("ORACLE_BUILD", os.path.join(_HERE, "_build"))
# ORACLE_SANITIZE=1: an AddressSanitizer + UndefinedBehaviorSanitizer build
# (its own file; the process must preload the ASan runtime).
_SANITIZE = os.environ.get("ORACLE_SANITIZE") == "1"
_LIB_PATH = os.path.join(_BUILD, "libism_oracle_san.so" if _SANITIZE else "libism_oracle.so")

FD_HANN_SINC = 0
FD_LAGRANGE = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    if _SANITIZE:
        cmd[1:1] = ["-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer",
                    "-fno-sanitize-recover=undefined"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        lib.oracle_rir.argtypes = [P, P, P, P, f64, f64, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, i64, P, P]
        lib.oracle_rir.restype = ctypes.c_int
        lib.oracle_auto_order.argtypes = [P, P, P, f64, f64, ctypes.c_int, i64]
        lib.oracle_auto_order.restype = ctypes.c_int
        lib.oracle_images.argtypes = [P, P, P, P, f64, f64, ctypes.c_int, P, P, P]
        lib.oracle_images.restype = i64
        lib.oracle_rir_batch.argtypes = [i64, P, P, P, P, P, P, P, P, ctypes.c_int]
        lib.oracle_rir_batch.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_hann_sinc_taps.argtypes = [f64, ctypes.c_int, P]
        lib.oracle_lagrange_taps.argtypes = [f64, ctypes.c_int, P]
        lib.oracle_convolve.argtypes = [P, i64, P, i64, P]
        lib.oracle_convolve_at.argtypes = [P, i64, P, i64, P, i64, P]
        lib.oracle_convolve_batch.argtypes = [i64, P, P, P, P, P, P, P, P, P, ctypes.c_int]
        lib.oracle_splitmix64.argtypes = [u64, u64]
        lib.oracle_splitmix64.restype = u64
        lib.oracle_gauss.argtypes = [u64, u64, u64, u64]
        lib.oracle_gauss.restype = f64
        lib.oracle_uniforms.argtypes = [u64, u64, u64, u64, i64, P, P]
        lib.oracle_add_noise.argtypes = [P, ctypes.c_int, i64, f64, u64, u64]
        lib.oracle_add_noise.restype = f64
        lib.oracle_frame.argtypes = [P, ctypes.c_int, i64, i64, ctypes.c_int, f64, u64, u64, P]
        lib.oracle_frame.restype = f64
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def rir(dims, beta, src, mic, fs, c, order, n_taps=81, fd_kind=FD_HANN_SINC, rir_len=4096,
        return_stats=False):
    """One RIR h[0..rir_len) (FP64) from the full (2N+1)^3 x 8 image lattice."""
    lib = _load()
    d, b, s, m = _f64(dims), _f64(beta), _f64(src), _f64(mic)
    h = np.zeros(int(rir_len), np.float64)
    st = np.zeros(3, np.int64)
    lib.oracle_rir(_p(d), _p(b), _p(s), _p(m), float(fs), float(c), int(order), int(n_taps),
                   int(fd_kind), int(rir_len), _p(h), _p(st))
    if return_stats:
        return h, {"images": int(st[0]), "contributing": int(st[1]), "taps": int(st[2])}
    return h


def auto_order(dims, src, mic, fs, c, n_taps, rir_len):
    """Order of the delay-limited image set (order < 0 in rir / rir_batch)."""
    lib = _load()
    return int(lib.oracle_auto_order(_p(_f64(dims)), _p(_f64(src)), _p(_f64(mic)), float(fs),
                                     float(c), int(n_taps), int(rir_len)))


def images(dims, beta, src, mic, fs, c, order):
    """All lattice images: dict of idx (n,6: u,v,w,l,m,n), d, tau, f, amp, k0."""
    lib = _load()
    n = 8 * (2 * int(order) + 1) ** 3
    idx = np.zeros((n, 6), np.int32)
    dtfa = np.zeros((n, 4), np.float64)
    k0 = np.zeros(n, np.int64)
    d, b, s, m = _f64(dims), _f64(beta), _f64(src), _f64(mic)
    cnt = lib.oracle_images(_p(d), _p(b), _p(s), _p(m), float(fs), float(c), int(order),
                            _p(idx), _p(dtfa), _p(k0))
    assert cnt == n
    return {"idx": idx, "d": dtfa[:, 0].copy(), "tau": dtfa[:, 1].copy(),
            "f": dtfa[:, 2].copy(), "amp": dtfa[:, 3].copy(), "k0": k0, "count": int(cnt)}


def rir_batch(rooms, n_threads=0):
    """RIRs for a list of room dicts (keys: dims, beta, src, mics (M,3), fs, c,
    order, n_taps, fd_kind, rir_len).  Returns (list of (M, Lh) arrays, stats
    array (n_rirs, 3)).  Parallel over RIRs with OpenMP."""
    lib = _load()
    room_f = np.zeros((len(rooms), 15), np.float64)
    room_i = np.zeros((len(rooms), 4), np.int32)
    room_len = np.zeros(len(rooms), np.int64)
    room_of, mics, offs = [], [], []
    off = 0
    for r, rm in enumerate(rooms):
        room_f[r, 0:3] = rm["dims"]
        room_f[r, 3:9] = rm["beta"]
        room_f[r, 9:12] = rm["src"]
        room_f[r, 12] = rm["fs"]
        room_f[r, 13] = rm["c"]
        room_i[r, 0] = rm["order"]
        room_i[r, 1] = rm.get("n_taps", 81)
        room_i[r, 2] = rm.get("fd_kind", FD_HANN_SINC)
        room_len[r] = rm["rir_len"]
        for mic in np.asarray(rm["mics"], np.float64).reshape(-1, 3):
            room_of.append(r)
            mics.append(mic)
            offs.append(off)
            off += int(rm["rir_len"])
    room_of = np.asarray(room_of, np.int32)
    mics = _f64(np.asarray(mics).reshape(-1, 3))
    offs = np.asarray(offs, np.int64)
    h = np.zeros(off, np.float64)
    stats = np.zeros((len(room_of), 3), np.int64)
    lib.oracle_rir_batch(len(room_of), _p(room_of), _p(room_f), _p(room_i), _p(room_len),
                         _p(mics), _p(h), _p(offs), _p(stats), int(n_threads))
    out, j = [], 0
    for rm in rooms:
        M = np.asarray(rm["mics"]).reshape(-1, 3).shape[0]
        L = int(rm["rir_len"])
        out.append(h[offs[j]:offs[j] + M * L].reshape(M, L))
        j += M
    return out, stats


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def hann_sinc_taps(f, n_taps=81):
    out = np.zeros(n_taps, np.float64)
    _load().oracle_hann_sinc_taps(float(f), int(n_taps), _p(out))
    return out


def lagrange_taps(D, n_taps=8):
    out = np.zeros(n_taps, np.float64)
    _load().oracle_lagrange_taps(float(D), int(n_taps), _p(out))
    return out


def convolve(h, s):
    """Full linear convolution (len(s) + len(h) - 1 samples), FP64."""
    h, s = _f64(h), _f64(s)
    y = np.zeros(len(s) + len(h) - 1, np.float64)
    _load().oracle_convolve(_p(h), len(h), _p(s), len(s), _p(y))
    return y


def convolve_at(h, s, ts):
    """Outputs y[t] for the listed t of the full linear convolution."""
    h, s = _f64(h), _f64(s)
    ts = np.ascontiguousarray(ts, np.int64)
    y = np.zeros(len(ts), np.float64)
    _load().oracle_convolve_at(_p(h), len(h), _p(s), len(s), _p(ts), len(ts), _p(y))
    return y


def convolve_batch(hs, srcs, n_threads=0):
    """hs: list (per room) of (M, Lh) arrays; srcs: list of 1-D sources.
    Returns a list of (M, Ts + Lh - 1) arrays.  OpenMP over (room, mic)."""
    lib = _load()
    room_of, h_off, h_len, y_off = [], [], [], []
    h_parts, s_parts, s_off, s_len = [], [], [], []
    ho = so = yo = 0
    for r, (H, s) in enumerate(zip(hs, srcs)):
        H = np.asarray(H, np.float64)
        s_off.append(so)
        s_len.append(len(s))
        s_parts.append(_f64(s))
        so += len(s)
        for m in range(H.shape[0]):
            room_of.append(r)
            h_off.append(ho)
            h_len.append(H.shape[1])
            y_off.append(yo)
            h_parts.append(H[m])
            ho += H.shape[1]
            yo += len(s) + H.shape[1] - 1
    hcat = _f64(np.concatenate(h_parts))
    scat = _f64(np.concatenate(s_parts))
    y = np.zeros(yo, np.float64)
    a = lambda x: np.ascontiguousarray(x, np.int64)
    room_of = np.asarray(room_of, np.int32)
    h_off, h_len, y_off, s_off, s_len = a(h_off), a(h_len), a(y_off), a(s_off), a(s_len)
    lib.oracle_convolve_batch(len(room_of), _p(room_of), _p(hcat), _p(h_off), _p(h_len),
                              _p(scat), _p(s_off), _p(s_len), _p(y), _p(y_off), int(n_threads))
    out, j = [], 0
    for H, s in zip(hs, srcs):
        M, L = np.asarray(H).shape
        T = len(s) + L - 1
        out.append(y[y_off[j]:y_off[j] + M * T].reshape(M, T))
        j += M
    return out


def splitmix64(state: int, i: int) -> int:
    return int(_load().oracle_splitmix64(state & (2**64 - 1), i & (2**64 - 1)))


def gauss(seed, room, mic, t) -> float:
    return float(_load().oracle_gauss(seed, room, mic, t))


def uniforms(seed, room, mic, k0, n):
    """u1, u2 of sample pairs k0 .. k0+n-1 of stream (room, mic)."""
    u1 = np.zeros(n, np.float64)
    u2 = np.zeros(n, np.float64)
    _load().oracle_uniforms(seed, room, mic, k0, n, _p(u1), _p(u2))
    return u1, u2


def frame(y, t0, frame_len, snr_db, seed, frame_id):
    """One training frame from a room's signals y (n_mics, y_len): the slice
    [t0, t0 + frame_len) (zero outside), plus noise at snr_db (NaN / inf =
    clean).  Returns (frame (n_mics, frame_len) FP64, sigma)."""
    lib = _load()
    y = np.ascontiguousarray(np.asarray(y, np.float64))
    if y.ndim == 1:
        y = y[None, :]
    out = np.zeros((y.shape[0], int(frame_len)), np.float64)
    sig = lib.oracle_frame(_p(y), int(y.shape[0]), int(y.shape[1]), int(t0), int(frame_len),
                           float(snr_db), int(seed), int(frame_id), _p(out))
    return out, float(sig)


def add_noise(y, snr_db, seed, room):
    """Adds the room's noise in place to y (M, T) FP64; returns sigma."""
    y = np.ascontiguousarray(y, np.float64)
    M, T = y.shape
    sigma = _load().oracle_add_noise(_p(y), M, T, float(snr_db), int(seed), int(room))
    return y, sigma
