"""Host-side checks of the C ABI (no GPU needed).

libism.so loads on a machine without a GPU, exports every function that
include/ism.h declares, rejects invalid arguments before touching the
device, and its serving layer reports (rather than hangs on) a device it
cannot use: the failure is made on the host (a device ordinal that does not
exist), never by faulting a GPU.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_13347_gb300 import _lib, build
    build.build()
    return _lib


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ism.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ism_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 13
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), f"libism.so does not export {n}"
    assert set(names) == set(lib.SIGNATURES), "binding signatures out of sync with ism.h"


def test_version_and_error_string(lib):
    L = lib.load()
    assert b"sm_103a" in L.ism_version()
    assert L.ism_last_error_string() is not None


def good_room(**kw):
    r = dict(dims=[5.0, 4.0, 3.0], beta=[0.8] * 6, src=[1.0, 1.0, 1.0],
             mics=[[2.0, 2.0, 2.0]], fs=16000.0, c=343.0, order=3, n_taps=81, fd_kind=0,
             rir_len=1024)
    r.update(kw)
    return r


BAD = {
    "source outside": dict(src=[6.0, 1.0, 1.0]),
    "source on wall": dict(src=[0.0, 1.0, 1.0]),
    "mic outside": dict(mics=[[2.0, 5.0, 1.0]]),
    "mic on source": dict(mics=[[1.0, 1.0, 1.0]]),
    "beta above 1": dict(beta=[0.8] * 5 + [1.2]),
    "beta negative": dict(beta=[-0.1] + [0.8] * 5),
    "even hann taps": dict(n_taps=80),
    "odd lagrange taps": dict(fd_kind=1, n_taps=7),
    "unknown filter": dict(fd_kind=5),
    "fs zero": dict(fs=0.0),
    "c negative": dict(c=-343.0),
    "auto order above 200": dict(dims=[0.5, 0.5, 0.5], src=[0.2, 0.2, 0.2],
                                 mics=[[0.3, 0.3, 0.3]], order=-1, rir_len=100000),
    "order too high": dict(order=201),
    "empty rir": dict(rir_len=0),
    "no mics": dict(mics=np.zeros((0, 3))),
    "nan dims": dict(dims=[float("nan"), 4.0, 3.0]),
}


BAD.update({
    "hann taps above 255": dict(n_taps=257),
    "lagrange taps above 32": dict(fd_kind=1, n_taps=34),
    "rir above 2^30": dict(rir_len=(1 << 30) + 1),
    "infinite fs": dict(fs=float("inf")),
    "nan beta": dict(beta=[0.8] * 5 + [float("nan")]),
    "nan mic": dict(mics=[[2.0, float("nan"), 2.0]]),
    "lattice delays beyond 8e6 samples": dict(dims=[20.0, 20.0, 20.0], order=200, fs=192000.0),
    "more than 65536 mics": dict(mics=np.tile([[2.0, 2.0, 2.0]], (65537, 1))),
})


def device_buffer(n):
    """A real device buffer where a GPU is present (so that a regression in
    the checks could never launch onto a stray pointer), else a pointer the
    library must never dereference."""
    import torch
    if torch.cuda.is_available():
        t = torch.zeros(n, device="cuda")
        return t, ctypes.c_void_p(t.data_ptr())
    return None, ctypes.c_void_p(0x1000)


@pytest.mark.parametrize("case", sorted(BAD))
def test_rir_batch_rejects_invalid_rooms(lib, case):
    L = lib.load()
    r = good_room(**BAD[case])
    arr, keep = lib.make_rooms([r])
    buf, ptr = device_buffer(1 << 16)
    st = L.ism_rir_batch(arr, 1, ptr, None, None)
    assert st == lib.ISM_ERR_INVALID_ARG, (case, st, lib.last_error())
    assert lib.last_error()


def documented_valid(r):
    """The room rules include/ism.h states for ism_rir_batch, restated (the
    delay-limited order by the header's formula; the 8e6-sample delay rule
    cannot fire on the rooms drawn below)."""
    d, b = np.asarray(r["dims"], float), np.asarray(r["beta"], float)
    s, mics = np.asarray(r["src"], float), np.asarray(r["mics"], float).reshape(-1, 3)
    if not np.all(np.isfinite(d) & (d > 0)) or not np.all((b >= 0) & (b <= 1)):
        return False
    inside = lambda p: bool(np.all((p > 0) & (p < d)))
    if not inside(s) or not 1 <= len(mics) <= 65536:
        return False
    for m in mics:
        if not inside(m) or float(np.sum((m - s) ** 2)) < 1e-12:
            return False
    fs, c, L, taps, kind = r["fs"], r["c"], r["rir_len"], r["n_taps"], r["fd_kind"]
    if not (fs > 0 and math.isfinite(fs) and c > 0 and math.isfinite(c)) or not 1 <= L <= 1 << 30:
        return False
    if kind == 0:
        if not (1 <= taps <= 255 and taps % 2 == 1):
            return False
    elif kind == 1:
        if not (2 <= taps <= 32 and taps % 2 == 0):
            return False
    else:
        return False
    order = r["order"]
    if order < 0:
        reach = (L + taps) * c / fs
        order = max(int(math.floor((reach + abs((1 - 2 * p) * s[a] - m[a])) / (2 * d[a])))
                    for m in mics for a in range(3) for p in (0, 1))
    return order <= 200


def test_room_checks_follow_the_documented_rules(lib):
    """Seeded random rooms, valid and invalid in every field (non-finite
    values, points on or past a wall, tap counts at and past each filter's
    limits, orders past 200, RIR lengths at 2^30): the library accepts
    exactly the rooms the header's rules accept (host-only call)."""
    L = lib.load()
    rng = np.random.default_rng(77)
    bad_f = [0.0, -1.0, float("nan"), float("inf")]
    n_ok = 0
    for _ in range(3000):
        r = good_room()
        pick = lambda p: rng.random() < p
        r["dims"] = list(rng.uniform(1, 10, 3))
        if pick(0.05):
            r["dims"][int(rng.integers(3))] = float(rng.choice(bad_f))
        r["beta"] = list(rng.uniform(0, 1, 6))
        if pick(0.05):
            r["beta"][int(rng.integers(6))] = float(rng.choice([-0.1, 1.1, float("nan")]))
        dims = np.nan_to_num(np.abs(np.asarray(r["dims"], float)), posinf=1.0) + 1e-9

        def point():
            p = rng.uniform(0.01, 0.99, 3) * dims
            if pick(0.05):
                a = int(rng.integers(3))
                p[a] = float(rng.choice([0.0, dims[a], -0.5, dims[a] + 0.5, float("nan")]))
            return p

        r["src"] = list(point())
        r["mics"] = np.array([point() for _ in range(int(rng.integers(0, 4)))]).reshape(-1, 3)
        if pick(0.03) and len(r["mics"]):
            r["mics"][0] = r["src"]
        r["fs"] = float(rng.uniform(8000, 48000)) if not pick(0.05) else float(rng.choice(bad_f))
        r["c"] = float(rng.uniform(300, 400)) if not pick(0.05) else float(rng.choice(bad_f))
        r["order"] = (int(rng.choice([-1, 0, 3, 15])) if not pick(0.2)
                      else int(rng.choice([-5, 200, 201, 250])))
        r["fd_kind"] = int(rng.choice([0, 1])) if not pick(0.05) else int(rng.choice([2, -1]))
        valid_taps = [1, 3, 9, 33, 81, 255] if r["fd_kind"] == 0 else [2, 8, 32]
        r["n_taps"] = (int(rng.choice(valid_taps)) if not pick(0.2)
                       else int(rng.choice([-1, 0, 2, 3, 34, 80, 256, 257])))
        r["rir_len"] = (int(rng.choice([1, 100, 5000])) if not pick(0.15)
                        else int(rng.choice([-5, 0, 60000, 1 << 30, (1 << 30) + 1])))
        if len(r["mics"]) == 0:
            continue  # an empty mic array needs a NULL pointer: covered by BAD
        arr, keep = lib.make_rooms([r])
        w = ctypes.c_int32(-7)
        st = L.ism_rir_tuned_window(arr, 1, None, ctypes.byref(w))
        want = documented_valid(r)
        assert st == (lib.ISM_OK if want else lib.ISM_ERR_INVALID_ARG), (r, st, lib.last_error())
        n_ok += want
    assert 500 < n_ok < 2500


def test_rir_batch_argument_errors(lib):
    L = lib.load()
    arr, keep = lib.make_rooms([good_room()])
    assert L.ism_rir_batch(arr, -1, ctypes.c_void_p(0x1000), None, None) == lib.ISM_ERR_INVALID_ARG
    assert L.ism_rir_batch(arr, 1, None, None, None) == lib.ISM_ERR_INVALID_ARG
    assert L.ism_rir_batch(None, 0, None, None, None) == lib.ISM_OK  # empty batch: no-op
    opts = lib.RirOpts(48, 0, None)  # window not a multiple of 32
    assert L.ism_rir_batch_ex(arr, 1, ctypes.c_void_p(0x1000), None, ctypes.byref(opts),
                              None) == lib.ISM_ERR_INVALID_ARG


def test_rir_batch_size(lib):
    rooms = [good_room(), good_room(mics=[[2, 2, 2], [3, 1, 1], [1, 3, 2]], rir_len=77)]
    assert lib.rir_batch_size(rooms) == (4, 1024 + 3 * 77)


def test_convolve_batch_argument_errors(lib):
    L = lib.load()
    jobs, _ = lib.conv_jobs([2], [100], [50])
    p = ctypes.c_void_p(0x1000)
    assert L.ism_convolve_batch(jobs, 1, p, p, p, 0, 7, None) == lib.ISM_ERR_INVALID_ARG
    assert L.ism_convolve_batch(jobs, 1, None, p, p, 0, 0, None) == lib.ISM_ERR_INVALID_ARG
    bad, _ = lib.conv_jobs([0], [100], [50])
    assert L.ism_convolve_batch(bad, 1, p, p, p, 0, 0, None) == lib.ISM_ERR_INVALID_ARG
    inf_snr, _ = lib.conv_jobs([1], [100], [50], snr_db=[float("inf")])
    assert L.ism_convolve_batch(inf_snr, 1, p, p, p, 0, 0, None) == lib.ISM_ERR_INVALID_ARG
    assert L.ism_convolve_batch(jobs, 0, p, p, p, 0, 0, None) == lib.ISM_OK


def conv_job_valid(n_mics, rir_len, src_len, offs, snr):
    """The job rules include/ism.h states for ism_convolve_batch, restated."""
    if not (1 <= n_mics <= 65536 and 1 <= rir_len <= 1 << 40 and 1 <= src_len <= 1 << 40):
        return False
    if min(offs) < 0 or not (math.isnan(snr) or math.isfinite(snr)):
        return False
    tiles = -(-n_mics // 8) * -(-(src_len + rir_len - 1) // 2048)
    return tiles <= (1 << 30) - 1


def test_convolve_job_checks_follow_the_documented_rules(lib):
    """Seeded random jobs at and past every documented limit (lengths up to
    2^63 - 1, mic counts past 65536, negative offsets, infinite SNRs, tile
    counts past 2^30): every job the rules reject is rejected before the
    device is touched.  Jobs the rules accept are submitted only where no GPU
    is present (the fake pointers are never dereferenced; the call then
    fails on the device, not on its arguments)."""
    import torch
    L = lib.load()
    gpu = torch.cuda.is_available()
    p = ctypes.c_void_p(0x1000)
    rng = np.random.default_rng(5)
    big = [1, 7, 2048, 1 << 20, 1 << 40, (1 << 40) + 1, (1 << 62), (1 << 63) - 1, 0, -1]
    n_valid = n_invalid = 0
    for _ in range(2000):
        n = int(rng.integers(1, 4))
        fields = []
        for _ in range(n):
            fields.append((int(rng.choice([1, 8, 9, 33, 65536, 65537, 0, -3])),
                           int(rng.choice(big)), int(rng.choice(big)),
                           [int(rng.choice([0, 5, 1 << 40, -1])) if rng.random() < 0.1 else 0
                            for _ in range(3)],
                           float(rng.choice([np.nan, 0.0, 30.0, 1e30, np.inf, -np.inf]))))
        jobs = (lib.ConvJob * n)()
        for J, (m, lh, ls, offs, snr) in zip(jobs, fields):
            J.n_mics, J.rir_len, J.src_len = m, lh, ls
            J.h_offset, J.src_offset, J.y_offset = offs
            J.snr_db = snr
        want = all(conv_job_valid(*f) for f in fields)
        if want and gpu:
            continue
        st = L.ism_convolve_batch(jobs, n, p, p, p, 0, int(rng.integers(0, 2)), None)
        if want:
            assert st != lib.ISM_ERR_INVALID_ARG, (fields, lib.last_error())
            n_valid += 1
        else:
            assert st == lib.ISM_ERR_INVALID_ARG, fields
            n_invalid += 1
    assert n_invalid > 500 and (gpu or n_valid > 20)


def test_frame_job_checks_follow_the_documented_rules(lib):
    """Seeded random frame jobs at and past the documented limits (mic
    counts past 65536, row lengths past 2^40, negative offsets, SNR -inf,
    frame lengths below 1): rejected exactly when the rules say so; jobs the
    rules accept are submitted only where no GPU is present."""
    import torch
    L = lib.load()
    gpu = torch.cuda.is_available()
    p = ctypes.c_void_p(0x1000)
    rng = np.random.default_rng(6)
    n_invalid = 0
    for _ in range(1000):
        m = int(rng.choice([1, 8, 65536, 65537, 0, -1]))
        yl = int(rng.choice([1, 1000, 1 << 40, (1 << 40) + 1, 0, -7]))
        yo, oo = (int(rng.choice([0, 9, -1])) for _ in range(2))
        snr = float(rng.choice([np.nan, 10.0, np.inf, -np.inf]))
        fl = int(rng.choice([1, 1024, 0, -2]))
        want = (1 <= m <= 65536 and 1 <= yl <= 1 << 40 and yo >= 0 and oo >= 0
                and snr != -np.inf and fl >= 1)
        if want and gpu:
            continue
        jobs = (lib.FrameJob * 1)()
        J = jobs[0]
        J.n_mics, J.y_len, J.y_offset, J.out_offset, J.t0, J.snr_db = m, yl, yo, oo, 0, snr
        st = L.ism_frames_batch(jobs, 1, fl, p, p, 0, None)
        if want:
            assert st != lib.ISM_ERR_INVALID_ARG, (m, yl, yo, oo, snr, fl, lib.last_error())
        else:
            assert st == lib.ISM_ERR_INVALID_ARG, (m, yl, yo, oo, snr, fl)
            n_invalid += 1
    assert n_invalid > 300


# --------------------------------------------------------------------------
# serving: host-side failure paths
# --------------------------------------------------------------------------

def make_request(lib, room, src):
    arr, keep = lib.make_rooms([room])
    rq = lib.Request()
    rq.room = arr[0]
    rq.src_host = src.ctypes.data
    rq.src_len = len(src)
    rq.snr_db = math.nan
    return rq, keep


def serve(lib, **kw):
    cfg = lib.ServeConfig()
    for k, v in kw.items():
        setattr(cfg, k, v)
    srv = ctypes.c_void_p()
    st = lib.load().ism_serve_create(ctypes.byref(cfg), ctypes.byref(srv))
    return st, srv


def test_serve_config_validation(lib):
    assert serve(lib, precision=9)[0] == lib.ISM_ERR_INVALID_ARG
    assert serve(lib, n_streams=17)[0] == lib.ISM_ERR_INVALID_ARG
    assert serve(lib, max_batch=-1)[0] == lib.ISM_ERR_INVALID_ARG


def test_serve_unusable_device_fails_requests(lib):
    """A device ordinal that does not exist: submits are accepted, the
    serving thread cannot select the device, and every request reports
    ISM_ERR_CUDA through wait/poll; nothing hangs."""
    L = lib.load()
    st, srv = serve(lib, device=97, max_queue=8)
    assert st == lib.ISM_OK
    src = np.ones(100, np.float32)
    tickets = []
    for _ in range(3):
        rq, keep = make_request(lib, good_room(), src)
        t = ctypes.c_uint64()
        assert L.ism_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)) == lib.ISM_OK
        tickets.append(t.value)
    res = lib.Result()
    for t in tickets:
        st = L.ism_serve_wait(srv, t, 30.0, ctypes.byref(res))
        assert st == lib.ISM_ERR_CUDA, (st, lib.last_error())
        assert "device 97" in lib.last_error()
        assert L.ism_serve_poll(srv, t, ctypes.byref(res)) == lib.ISM_ERR_CUDA
        assert L.ism_serve_release(srv, t) == lib.ISM_OK
        assert L.ism_serve_poll(srv, t, ctypes.byref(res)) == lib.ISM_ERR_UNKNOWN_TICKET
        assert L.ism_serve_release(srv, t) == lib.ISM_ERR_UNKNOWN_TICKET
    stats = lib.ServeStats()
    assert L.ism_serve_stats_get(srv, ctypes.byref(stats)) == lib.ISM_OK
    assert stats.submitted == 3 and stats.queued == 0
    assert L.ism_serve_destroy(srv) == lib.ISM_OK


def test_serve_admission_limits(lib):
    """BUSY for a request larger than the memory budget and for more
    outstanding (unreleased) requests than max_queue; INVALID_ARG for a bad
    room or an empty source."""
    L = lib.load()
    st, srv = serve(lib, device=97, max_queue=2, max_hbm_bytes=1 << 20)
    assert st == lib.ISM_OK
    t = ctypes.c_uint64()
    big = np.ones(400000, np.float32)  # > 1 MiB with outputs
    rq, keep = make_request(lib, good_room(), big)
    assert L.ism_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)) == lib.ISM_ERR_BUSY
    small = np.ones(50, np.float32)
    held = []
    for _ in range(2):
        rq, keep = make_request(lib, good_room(rir_len=64), small)
        assert L.ism_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)) == lib.ISM_OK
        held.append(t.value)
    rq, keep = make_request(lib, good_room(rir_len=64), small)
    assert L.ism_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)) == lib.ISM_ERR_BUSY
    rq, keep = make_request(lib, good_room(src=[9.0, 1.0, 1.0]), small)
    assert L.ism_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)) == lib.ISM_ERR_INVALID_ARG
    rq, keep = make_request(lib, good_room(), small)
    rq.src_len = 0
    assert L.ism_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)) == lib.ISM_ERR_INVALID_ARG
    res = lib.Result()
    for h in held:
        L.ism_serve_wait(srv, h, 30.0, ctypes.byref(res))
        assert L.ism_serve_release(srv, h) == lib.ISM_OK
    rq, keep = make_request(lib, good_room(rir_len=64), small)
    assert L.ism_serve_submit(srv, ctypes.byref(rq), ctypes.byref(t)) == lib.ISM_OK
    stats = lib.ServeStats()
    L.ism_serve_stats_get(srv, ctypes.byref(stats))
    assert stats.rejected_busy == 2
    assert L.ism_serve_destroy(srv) == lib.ISM_OK


def test_serve_wait_on_unknown_ticket(lib):
    L = lib.load()
    st, srv = serve(lib, device=97)
    res = lib.Result()
    assert L.ism_serve_wait(srv, 12345, 0.01, ctypes.byref(res)) == lib.ISM_ERR_UNKNOWN_TICKET
    assert L.ism_serve_destroy(srv) == lib.ISM_OK


def test_frames_batch_argument_errors(lib):
    L = lib.load()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: validation comes first
    jobs, n = lib.frame_jobs([0], [100], [2], [0], 64)
    assert L.ism_frames_batch(jobs, 1, 64, None, fake, 0, None) == lib.ISM_ERR_INVALID_ARG
    assert L.ism_frames_batch(jobs, 1, 0, fake, fake, 0, None) == lib.ISM_ERR_INVALID_ARG
    assert L.ism_frames_batch(jobs, -1, 64, fake, fake, 0, None) == lib.ISM_ERR_INVALID_ARG
    assert L.ism_frames_batch(None, 0, 64, None, None, 0, None) == lib.ISM_OK
    for field, val in (("n_mics", 0), ("y_len", 0), ("y_offset", -1), ("out_offset", -1),
                       ("snr_db", -math.inf)):
        jobs, n = lib.frame_jobs([0], [100], [2], [0], 64)
        setattr(jobs[0], field, val)
        assert L.ism_frames_batch(jobs, 1, 64, fake, fake, 0, None) == lib.ISM_ERR_INVALID_ARG, field
        assert lib.last_error()


def test_dataset_batch_argument_errors(lib):
    L = lib.load()
    arr, keep = lib.make_rooms([good_room()])
    src = np.zeros(100, np.float32)
    y = np.zeros(8 * 2000, np.float32)
    lens = np.array([100], np.int64)
    P = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    ok_args = [arr, 1, P(src), P(lens), None, None, 0, 0, 1, P(y), None, None, None, 0]

    def call(**kw):
        a = list(ok_args)
        names = ["rooms", "n", "src", "lens", "so", "snr", "seed", "base", "prec", "y", "yo", "h",
                 "ho", "chunk"]
        for k, v in kw.items():
            a[names.index(k)] = v
        return L.ism_dataset_batch(*a)

    assert call(src=None) == lib.ISM_ERR_INVALID_ARG
    assert call(y=None) == lib.ISM_ERR_INVALID_ARG
    assert call(lens=None) == lib.ISM_ERR_INVALID_ARG
    assert call(prec=7) == lib.ISM_ERR_INVALID_ARG
    assert call(chunk=-1) == lib.ISM_ERR_INVALID_ARG
    assert call(n=0) == lib.ISM_OK
    bad = np.array([0], np.int64)
    assert call(lens=P(bad)) == lib.ISM_ERR_INVALID_ARG
    arr2, keep2 = lib.make_rooms([good_room(src=[9.0, 1.0, 1.0])])
    assert call(rooms=arr2) == lib.ISM_ERR_INVALID_ARG
    assert lib.last_error()


def test_debug_inject_arguments(lib):
    """The fault-injection switch is host state only: unknown kinds are
    rejected, 0 cancels a pending injection."""
    L = lib.load()
    assert L.ism_debug_inject(99) == lib.ISM_ERR_INVALID_ARG
    assert "unknown injection" in lib.last_error()
    assert L.ism_debug_inject(lib.INJECT_CONV_WAIT) == lib.ISM_OK
    assert L.ism_debug_inject(0) == lib.ISM_OK


def test_tuned_window_reads_the_cache_file(lib, tmp_path, monkeypatch):
    """The autotuner's cache file (host only): a bucket that is not tuned
    reads as window 0; a line for the call's bucket -- variant, filter kinds
    (bit mask), Hann and Lagrange tap counts, largest order, sampling rate,
    ceil(log2 longest RIR), floor(log2 RIR count) -- gives its window."""
    L = lib.load()
    room = good_room(rir_len=1000, order=3)
    arr, keep = lib.make_rooms([room])
    w = ctypes.c_int32(-5)
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("ISM_TUNE_CACHE", str(path))
    assert L.ism_rir_tuned_window(arr, 1, None, ctypes.byref(w)) == lib.ISM_OK
    assert w.value == 0
    path2 = tmp_path / "tune2.txt"
    path2.write_text("ism-tune 1 0 1 81 0 3 16000 10 0 768 0.5\n"
                     "garbage line\n"
                     "ism-tune 1 0 1 81 0 3 16000 10 1 512 0.5\n")
    monkeypatch.setenv("ISM_TUNE_CACHE", str(path2))
    assert L.ism_rir_tuned_window(arr, 1, None, ctypes.byref(w)) == lib.ISM_OK
    assert w.value == 768
    bad = dict(room, beta=[2.0] * 6)
    arr2, keep2 = lib.make_rooms([bad])
    assert L.ism_rir_tuned_window(arr2, 1, None, ctypes.byref(w)) == lib.ISM_ERR_INVALID_ARG


def test_bounds_flags_need_the_checked_build(lib):
    """ism_debug_bounds answers only in the bounds-checked build (host-side
    in the normal one: no device call)."""
    import os as _os
    if "checked" in _os.environ.get("ISM_LIB", ""):
        pytest.skip("bounds-checked library loaded")
    f = ctypes.c_uint32(7)
    assert lib.load().ism_debug_bounds(ctypes.byref(f)) == lib.ISM_ERR_INVALID_ARG
    assert "bounds-checked" in lib.last_error()
