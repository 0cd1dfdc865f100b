"""ctypes binding of libism.so (include/ism.h).

Argument marshalling only: every step of the RIR and convolution path runs
in the library's CUDA kernels.  torch supplies device memory and streams.
If libism.so is missing or cannot be loaded this module raises; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# ISM_LIB selects another build of the library, e.g. the bounds-checked
# libism_checked.so (a file name is taken relative to this package)
LIB_PATH = os.path.join(HERE, os.environ.get("ISM_LIB", "libism.so"))

ISM_OK, ISM_PENDING = 0, 1
ISM_ERR_INVALID_ARG, ISM_ERR_OUT_OF_MEMORY, ISM_ERR_BUSY = 2, 3, 4
ISM_ERR_TIMEOUT, ISM_ERR_CUDA, ISM_ERR_INTERNAL, ISM_ERR_UNKNOWN_TICKET = 5, 6, 7, 8
INJECT_CONV_WAIT = 1
INJECT_SERVE_ALLOC = 2
WINDOW_TUNE = -1
FD_HANN_SINC, FD_LAGRANGE = 0, 1
RIR_SPARSE, RIR_DIRECT = 0, 1
F32, BF16X3 = 0, 1

c_i32, c_i64, c_u64, c_f32, c_f64, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_float, ctypes.c_double, ctypes.c_void_p)


class Room(ctypes.Structure):
    _fields_ = [("dims", c_f64 * 3), ("beta", c_f64 * 6), ("src", c_f64 * 3), ("mics", c_vp),
                ("n_mics", c_i32), ("order", c_i32), ("fs", c_f64), ("c", c_f64),
                ("n_taps", c_i32), ("fd_kind", c_i32), ("rir_len", c_i64)]


class RirOpts(ctypes.Structure):
    _fields_ = [("window", c_i32), ("per_room", c_i32), ("stats_dev", c_vp), ("variant", c_i32),
                ("reserved", c_i32)]


class ConvJob(ctypes.Structure):
    _fields_ = [("n_mics", c_i32), ("reserved", c_i32), ("rir_len", c_i64), ("src_len", c_i64),
                ("h_offset", c_i64), ("src_offset", c_i64), ("y_offset", c_i64),
                ("snr_db", c_f32), ("reserved2", c_i32), ("noise_id", c_u64)]


class FrameJob(ctypes.Structure):
    _fields_ = [("y_offset", c_i64), ("y_len", c_i64), ("t0", c_i64), ("out_offset", c_i64),
                ("noise_id", c_u64), ("n_mics", c_i32), ("snr_db", c_f32)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("max_hbm_bytes", c_i64), ("max_batch", c_i32), ("n_streams", c_i32),
                ("precision", c_i32), ("max_queue", c_i32), ("seed", c_u64), ("device", c_i32),
                ("reserved", c_i32)]


class Request(ctypes.Structure):
    _fields_ = [("room", Room), ("src_host", c_vp), ("src_len", c_i64), ("snr_db", c_f32),
                ("reserved", c_i32), ("noise_id", c_u64)]


class Result(ctypes.Structure):
    _fields_ = [("h_dev", c_vp), ("y_dev", c_vp), ("n_mics", c_i32), ("reserved", c_i32),
                ("rir_len", c_i64), ("y_len", c_i64), ("queue_s", c_f64), ("latency_s", c_f64)]


class PlanConfig(ctypes.Structure):
    _fields_ = [("precision", c_i32), ("window", c_i32), ("max_order", c_i32),
                ("variant", c_i32), ("seed", c_u64)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, c_i64) for n in ("submitted", "completed", "rejected_busy", "batches",
                                     "queued", "in_flight", "bytes_in_use", "bytes_peak", "taps",
                                     "mic_samples", "launch_host_ns", "batch_device_ns")]


# every symbol include/ism.h declares, with its ctypes signature
SIGNATURES = {
    "ism_rir_batch": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp]),
    "ism_rir_batch_ex": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "ism_rir_batch_size": (c_i32, [c_vp, c_i64, c_vp, c_vp]),
    "ism_rir_batch_noalloc": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp]),
    "ism_rir_filter_terms": (c_i32, [c_i32, c_i32, c_vp]),
    "ism_rir_tuned_window": (c_i32, [c_vp, c_i64, c_vp, c_vp]),
    "ism_convolve_batch": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp, c_u64, c_i32, c_vp]),
    "ism_frames_batch": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_vp, c_u64, c_vp]),
    "ism_dataset_batch": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_u64, c_u64, c_i32, c_vp,
                                  c_vp, c_vp, c_vp, c_i64]),
    "ism_plan_create": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "ism_plan_run": (c_i32, [c_vp, c_vp, c_vp, c_u64, c_vp]),
    "ism_plan_destroy": (c_i32, [c_vp]),
    "ism_serve_create": (c_i32, [c_vp, c_vp]),
    "ism_serve_submit": (c_i32, [c_vp, c_vp, c_vp]),
    "ism_serve_poll": (c_i32, [c_vp, c_u64, c_vp]),
    "ism_serve_wait": (c_i32, [c_vp, c_u64, c_f64, c_vp]),
    "ism_serve_release": (c_i32, [c_vp, c_u64]),
    "ism_serve_copy": (c_i32, [c_vp, c_u64, c_vp, c_vp, c_vp]),
    "ism_serve_stats_get": (c_i32, [c_vp, c_vp]),
    "ism_serve_destroy": (c_i32, [c_vp]),
    "ism_stream_status": (c_i32, [c_vp]),
    "ism_debug_inject": (c_i32, [c_i32]),
    "ism_debug_bounds": (c_i32, [c_vp]),
    "ism_last_error_string": (ctypes.c_char_p, []),
    "ism_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


class IsmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ism status {status}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Loads libism.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_2104_13347_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def last_error() -> str:
    return load().ism_last_error_string().decode()


def check(status: int):
    if status != ISM_OK:
        raise IsmError(status, last_error())
    return status


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_rooms(rooms):
    """Room dicts (dims, beta, src, mics (M,3), fs, c, order, n_taps,
    fd_kind, rir_len) -> (ctypes array, arrays kept alive)."""
    arr = (Room * len(rooms))()
    keep = []
    for i, r in enumerate(rooms):
        mics = np.ascontiguousarray(np.asarray(r["mics"], np.float64).reshape(-1, 3))
        keep.append(mics)
        R = arr[i]
        R.dims[:] = [float(x) for x in r["dims"]]
        R.beta[:] = [float(x) for x in r["beta"]]
        R.src[:] = [float(x) for x in r["src"]]
        R.mics = mics.ctypes.data
        R.n_mics = mics.shape[0]
        R.order = int(r["order"])
        R.fs = float(r["fs"])
        R.c = float(r["c"])
        R.n_taps = int(r.get("n_taps", 81))
        R.fd_kind = int(r.get("fd_kind", FD_HANN_SINC))
        R.rir_len = int(r["rir_len"])
    return arr, keep


def rir_batch_size(rooms):
    arr, keep = make_rooms(rooms)
    nr, hl = c_i64(), c_i64()
    check(load().ism_rir_batch_size(arr, len(rooms), ctypes.byref(nr), ctypes.byref(hl)))
    return nr.value, hl.value


def rir_tuned_window(rooms, variant=RIR_SPARSE):
    """The window rir_batch(..., window=WINDOW_TUNE) uses for these rooms,
    or 0 if their bucket is not tuned yet (host only)."""
    if isinstance(rooms, PreparedRooms):
        arr, n = rooms.arr, rooms.n
    else:
        arr, keep = make_rooms(rooms)
        n = len(rooms)
    opts = RirOpts(0, 0, None, int(variant), 0)
    w = c_i32()
    check(load().ism_rir_tuned_window(arr, n, ctypes.byref(opts), ctypes.byref(w)))
    return w.value


def rir_filter_terms(fd_kind, n_taps):
    """Chebyshev terms P the sparse path uses for a filter (0 = direct path)."""
    n = c_i32()
    check(load().ism_rir_filter_terms(int(fd_kind), int(n_taps), ctypes.byref(n)))
    return n.value


class PreparedRooms:
    """Rooms marshalled once into the C layout (reuse across calls)."""

    def __init__(self, rooms):
        self.arr, self.keep = make_rooms(rooms)
        self.n = len(rooms)
        self.n_rirs, self.h_len = rir_batch_size(rooms)


def rir_batch(rooms, h=None, h_offsets=None, window=0, per_room=False, stats=None, stream=None,
              variant=RIR_SPARSE):
    """ism_rir_batch_ex: RIRs of the rooms (room dicts or PreparedRooms) into
    h (a float32 CUDA tensor; allocated packed if None).  stats: optional
    int64 CUDA tensor (2 per RIR), accumulated.  variant: RIR_SPARSE
    (default) or RIR_DIRECT.  Returns h."""
    import torch
    lib = load()
    if isinstance(rooms, PreparedRooms):
        arr, keep = rooms.arr, [rooms.keep]
    else:
        arr, keep = make_rooms(rooms)
    if h is None:
        hl = rooms.h_len if isinstance(rooms, PreparedRooms) else rir_batch_size(rooms)[1]
        h = torch.empty(hl, dtype=torch.float32, device="cuda")
    assert h.dtype == torch.float32 and h.is_cuda and h.is_contiguous()
    offs = None
    if h_offsets is not None:
        offs = np.ascontiguousarray(h_offsets, np.int64)
        keep.append(offs)
    opts = RirOpts(int(window), int(bool(per_room)),
                   stats.data_ptr() if stats is not None else None, int(variant), 0)
    check(lib.ism_rir_batch_ex(arr, len(arr), c_vp(h.data_ptr()),
                               offs.ctypes.data if offs is not None else None,
                               ctypes.byref(opts), _stream_ptr(stream)))
    return h


def _rir_extent(rooms, offs):
    """Elements of h a RIR batch writes: the packed length, or with explicit
    offsets the end of the farthest RIR."""
    if isinstance(rooms, PreparedRooms):
        if offs is None:
            return rooms.h_len
        lens = [int(rooms.arr[i].rir_len) for i in range(rooms.n)
                for _ in range(int(rooms.arr[i].n_mics))]
    else:
        if offs is None:
            return rir_batch_size(rooms)[1]
        lens = [int(r["rir_len"]) for r in rooms
                for _ in range(np.asarray(r["mics"]).reshape(-1, 3).shape[0])]
    if len(offs) != len(lens):
        raise ValueError(f"h_offsets has {len(offs)} entries for {len(lens)} RIRs")
    return max((int(o) + L for o, L in zip(offs, lens)), default=0)


def rir_batch_noalloc(rooms, h, h_offsets=None, stream=None):
    """ism_rir_batch_noalloc: as rir_batch (room dicts or PreparedRooms) into
    an existing contiguous float32 CUDA tensor h that holds every RIR,
    through the entry point that allocates nothing."""
    import torch
    lib = load()
    if isinstance(rooms, PreparedRooms):
        arr, keep, n = rooms.arr, [rooms.keep], rooms.n
    else:
        arr, keep = make_rooms(rooms)
        n = len(rooms)
    if not (isinstance(h, torch.Tensor) and h.dtype == torch.float32 and h.is_cuda
            and h.is_contiguous()):
        raise ValueError("h must be a contiguous float32 CUDA tensor")
    offs = None
    if h_offsets is not None:
        offs = np.ascontiguousarray(h_offsets, np.int64)
        keep.append(offs)
    need = _rir_extent(rooms, offs)
    if h.numel() < need:
        raise ValueError(f"h holds {h.numel()} floats, the batch writes {need}")
    check(lib.ism_rir_batch_noalloc(arr, n, c_vp(h.data_ptr()),
                                    offs.ctypes.data if offs is not None else None,
                                    _stream_ptr(stream)))
    return h


def stream_status(stream=None):
    """ism_stream_status: waits for the stream's calls that hold a status
    cell and raises IsmError (ISM_ERR_INTERNAL) if a kernel of one of them
    reported an error since the last report."""
    check(load().ism_stream_status(_stream_ptr(stream)))


def debug_bounds():
    """ism_debug_bounds: the out-of-range bits the kernels of a bounds-checked
    build recorded since the last call (cleared), or None for the normal
    build."""
    f = ctypes.c_uint32()
    st = load().ism_debug_bounds(ctypes.byref(f))
    if st == ISM_ERR_INVALID_ARG:
        return None
    check(st)
    return f.value


def debug_inject(what=INJECT_CONV_WAIT):
    """ism_debug_inject: test aid that makes the next split-BF16 convolution
    launch stop on a bounded wait nothing ends (0 cancels)."""
    check(load().ism_debug_inject(int(what)))


def conv_jobs(rooms_mics, rir_lens, src_lens, snr_db=None, noise_ids=None, h_offsets=None,
              src_offsets=None, y_offsets=None):
    """Builds the ism_conv_job array for a packed batch: room i has
    rooms_mics[i] RIRs of rir_lens[i] samples and a source of src_lens[i]
    samples; outputs are packed (mic-major within a room).  Returns
    (jobs ctypes array, packed y length)."""
    n = len(rooms_mics)
    jobs = (ConvJob * n)()
    ho = so = yo = 0
    for i in range(n):
        M, L, T = int(rooms_mics[i]), int(rir_lens[i]), int(src_lens[i])
        J = jobs[i]
        J.n_mics, J.rir_len, J.src_len = M, L, T
        J.h_offset = ho if h_offsets is None else int(h_offsets[i])
        J.src_offset = so if src_offsets is None else int(src_offsets[i])
        J.y_offset = yo if y_offsets is None else int(y_offsets[i])
        J.snr_db = math.nan if snr_db is None else float(snr_db[i])
        J.noise_id = i if noise_ids is None else int(noise_ids[i])
        ho += M * L
        so += T
        yo += M * (T + L - 1)
    return jobs, yo


def convolve_batch(jobs, h, src, y, seed=0, precision=F32, stream=None):
    """ism_convolve_batch over a ConvJob array (see conv_jobs)."""
    check(load().ism_convolve_batch(jobs, len(jobs), c_vp(h.data_ptr()), c_vp(src.data_ptr()),
                                    c_vp(y.data_ptr()), c_u64(seed), int(precision),
                                    _stream_ptr(stream)))
    return y


def frame_jobs(y_offsets, y_lens, n_mics, t0s, frame_len, snr_db=None, noise_ids=None):
    """Builds the ism_frame_job array of a batch of frames: frame i reads the
    room whose signals start at y_offsets[i] (n_mics[i] rows of y_lens[i]
    samples) from sample t0s[i]; outputs are packed (frame-major, then
    mic-major).  Returns (jobs ctypes array, packed output length)."""
    n = len(t0s)
    jobs = (FrameJob * n)()
    off = 0
    for i in range(n):
        J = jobs[i]
        J.y_offset, J.y_len, J.t0 = int(y_offsets[i]), int(y_lens[i]), int(t0s[i])
        J.n_mics = int(n_mics[i])
        J.out_offset = off
        J.snr_db = math.nan if snr_db is None else float(snr_db[i])
        J.noise_id = i if noise_ids is None else int(noise_ids[i])
        off += J.n_mics * int(frame_len)
    return jobs, off


def frames_batch(jobs, frame_len, y, out, seed=0, stream=None):
    """ism_frames_batch over a FrameJob array (see frame_jobs)."""
    check(load().ism_frames_batch(jobs, len(jobs), int(frame_len), c_vp(y.data_ptr()),
                                  c_vp(out.data_ptr()), c_u64(seed), _stream_ptr(stream)))
    return out


def dataset_batch(rooms, src_host, src_lens, y_host, snr_db=None, seed=0, noise_id_base=0,
                  precision=BF16X3, h_host=None, chunk_rooms=0):
    """ism_dataset_batch: RIRs, convolution and noise with host buffers.
    rooms: room dicts or PreparedRooms; src_host: float32 sources packed in
    room order (a CPU tensor, page-locked for overlapped copies, or a numpy
    array); src_lens: samples per room; y_host (and optional h_host): CPU
    float32 outputs, packed.  Returns y_host."""
    import torch
    lib = load()
    if isinstance(rooms, PreparedRooms):
        arr, n = rooms.arr, rooms.n
    else:
        arr, keep = make_rooms(rooms)
        n = len(rooms)
    lens = np.ascontiguousarray(np.asarray(src_lens, np.int64))
    snr = None if snr_db is None else np.ascontiguousarray(np.asarray(snr_db, np.float32))

    def ptr(x):
        if x is None:
            return None
        if isinstance(x, torch.Tensor):
            assert x.device.type == "cpu" and x.dtype == torch.float32 and x.is_contiguous()
            return c_vp(x.data_ptr())
        assert x.dtype == np.float32 and x.flags["C_CONTIGUOUS"]
        return c_vp(x.ctypes.data)

    check(lib.ism_dataset_batch(arr, n, ptr(src_host), c_vp(lens.ctypes.data), None,
                                None if snr is None else c_vp(snr.ctypes.data), c_u64(seed),
                                c_u64(noise_id_base), int(precision), ptr(y_host), None,
                                ptr(h_host), None, int(chunk_rooms)))
    return y_host


class Plan:
    """ism_plan_*: the dataset step of a fixed batch shape captured into CUDA
    graphs and replayed (argument marshalling only).  h, src, y: the
    caller's float32 CUDA tensors (packed; src and y None for a plan of RIRs
    only), kept alive by the plan."""

    def __init__(self, rooms, h, src=None, y=None, src_lens=None, precision=BF16X3, window=0,
                 max_order=0, variant=RIR_SPARSE, seed=0):
        self._lib = load()
        arr, keep = (rooms.arr, [rooms.keep]) if isinstance(rooms, PreparedRooms) else \
            make_rooms(rooms)
        n = len(arr)
        for t in (h, src, y):
            if t is not None:
                assert t.dtype.is_floating_point and t.is_cuda and t.is_contiguous()
        lens = None
        if src_lens is not None:
            lens = np.ascontiguousarray(np.asarray(src_lens, np.int64))
            assert src is not None and y is not None and len(lens) == n
        cfg = PlanConfig(int(precision), int(window), int(max_order), int(variant), int(seed))
        self._h = c_vp()
        self._bufs = (h, src, y)
        check(self._lib.ism_plan_create(arr, n, None if lens is None else c_vp(lens.ctypes.data),
                                        ctypes.byref(cfg), c_vp(h.data_ptr()),
                                        None if src is None else c_vp(src.data_ptr()),
                                        None if y is None else c_vp(y.data_ptr()),
                                        ctypes.byref(self._h)))

    def run(self, rooms, snr_db=None, noise_id_base=0, stream=None):
        arr, keep = (rooms.arr, [rooms.keep]) if isinstance(rooms, PreparedRooms) else \
            make_rooms(rooms)
        snr = None if snr_db is None else np.ascontiguousarray(np.asarray(snr_db, np.float32))
        check(self._lib.ism_plan_run(self._h, arr, None if snr is None else c_vp(snr.ctypes.data),
                                     c_u64(noise_id_base), _stream_ptr(stream)))

    def close(self):
        if self._h:
            check(self._lib.ism_plan_destroy(self._h))
            self._h = c_vp()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class PreparedRequest:
    """A marshalled serving request (see Server.request)."""

    __slots__ = ("rq", "keep")

    def __init__(self, rq, keep):
        self.rq = rq
        self.keep = keep


class Server:
    """ism_serve_*: continuous-batching server (argument marshalling only)."""

    def __init__(self, max_hbm_bytes=0, max_batch=0, n_streams=0, precision=F32, max_queue=0,
                 seed=0, device=None):
        import torch
        self._lib = load()
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else 0
        cfg = ServeConfig(int(max_hbm_bytes), int(max_batch), int(n_streams), int(precision),
                          int(max_queue), int(seed), int(device), 0)
        self._h = c_vp()
        check(self._lib.ism_serve_create(ctypes.byref(cfg), ctypes.byref(self._h)))

    @staticmethod
    def request(room, src, snr_db=math.nan, noise_id=0):
        """Marshals one room dict and its float32 source into a request that
        submit() takes as is (argument marshalling only; the server copies
        the source when the request is submitted)."""
        arr, keep = make_rooms([room])
        src = np.ascontiguousarray(src, np.float32)
        rq = Request()
        rq.room = arr[0]
        rq.src_host = src.ctypes.data
        rq.src_len = len(src)
        rq.snr_db = float(snr_db)
        rq.noise_id = int(noise_id)
        return PreparedRequest(rq, (arr, keep, src))

    def submit(self, room, src=None, snr_db=math.nan, noise_id=0):
        """Submits one room dict and its float32 source, or a request made by
        request(); returns the ticket (raises IsmError with status
        ISM_ERR_BUSY when not admitted)."""
        if not isinstance(room, PreparedRequest):
            room = self.request(room, src, snr_db, noise_id)
        t = c_u64()
        check(self._lib.ism_serve_submit(self._h, ctypes.byref(room.rq), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        res = Result()
        st = self._lib.ism_serve_poll(self._h, c_u64(ticket), ctypes.byref(res))
        if st == ISM_PENDING:
            return None
        check(st)
        return res

    def wait(self, ticket, timeout_s=60.0):
        res = Result()
        check(self._lib.ism_serve_wait(self._h, c_u64(ticket), float(timeout_s),
                                       ctypes.byref(res)))
        return res

    def copy(self, ticket, h_out=None, y_out=None, stream=None):
        check(self._lib.ism_serve_copy(self._h, c_u64(ticket),
                                       c_vp(h_out.data_ptr()) if h_out is not None else None,
                                       c_vp(y_out.data_ptr()) if y_out is not None else None,
                                       _stream_ptr(stream)))

    def release(self, ticket):
        check(self._lib.ism_serve_release(self._h, c_u64(ticket)))

    def stats(self):
        s = ServeStats()
        check(self._lib.ism_serve_stats_get(self._h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in ServeStats._fields_}

    def close(self):
        if self._h:
            check(self._lib.ism_serve_destroy(self._h))
            self._h = c_vp()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
