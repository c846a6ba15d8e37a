"""Thin ctypes binding over libscpl's C ABI (include/scpl.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (torch supplies device memory
and streams), host buffers are numpy arrays or CPU tensors.  The library is
loaded on first use; a missing library raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libscpl.so")
_lib = None

(SCPL_OK, SCPL_EINVAL, SCPL_ENOMEM, SCPL_ECUDA, SCPL_ETIMEOUT, SCPL_EOVERFLOW,
 SCPL_ECANCELED) = range(7)
STATUS_NAMES = {0: "SCPL_OK", 1: "SCPL_EINVAL", 2: "SCPL_ENOMEM", 3: "SCPL_ECUDA",
                4: "SCPL_ETIMEOUT", 5: "SCPL_EOVERFLOW", 6: "SCPL_ECANCELED"}

# every symbol the header declares, with (restype, argtypes)
_P, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double


class Params(ctypes.Structure):
    """scpl_params (Sec. 3.2 alpha, Sec. 3.3 weights, buffer cap and mode, and
    the weight of the forward terms in the seam cost)."""
    _fields_ = [("alpha", ctypes.c_double), ("wg", ctypes.c_int), ("wm", ctypes.c_int),
                ("t_max", ctypes.c_int), ("use_buffer", ctypes.c_int),
                ("maxval_mode", ctypes.c_int), ("wf", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n_buffers", ctypes.c_int), ("iterations_max", ctypes.c_int),
                ("iterations_total", ctypes.c_longlong), ("carved_px", ctypes.c_double),
                ("n_kernels", ctypes.c_int), ("kernel", KernelStat * 8),
                ("launches", ctypes.c_longlong)]


class Job(ctypes.Structure):
    """scpl_job: one clip to retarget in a batch or through a server."""
    _fields_ = [("frames", ctypes.c_void_p), ("T", ctypes.c_int), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("target_W", ctypes.c_int), ("target_H", ctypes.c_int),
                ("k", ctypes.c_int), ("on_host", ctypes.c_int), ("out", ctypes.c_void_p),
                ("buffer_starts", ctypes.c_void_p), ("n_buffers", ctypes.c_int),
                ("status", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("queued", ctypes.c_int), ("active", ctypes.c_int),
                ("scan_waves", ctypes.c_longlong), ("groups", ctypes.c_longlong),
                ("chunks", ctypes.c_longlong), ("graphs_built", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("reserved_bytes", ctypes.c_size_t),
                ("peak_reserved_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("cancelled", ctypes.c_longlong)]


class Tuning(ctypes.Structure):
    """scpl_tuning: the kernel choices for one frame size and their times."""
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("dpc_halo", ctypes.c_int),
                ("dpc_warps", ctypes.c_int), ("dpc_lane_cols", ctypes.c_int),
                ("update_rows", ctypes.c_int),
                ("dp_us", ctypes.c_float * 7), ("up_us", ctypes.c_float * 3)]


_LL = ctypes.c_longlong
SIGNATURES = {
    "scpl_default_params": (None, [ctypes.POINTER(Params)]),
    "scpl_create": (_I, [ctypes.POINTER(Params), _P, ctypes.POINTER(_P)]),
    "scpl_set_stream": (_I, [_P, _P]),
    "scpl_destroy": (None, [_P]),
    "scpl_last_error": (ctypes.c_char_p, [_P]),
    "scpl_energy": (_I, [_P, _P, _I, _I, _I, _P]),
    "scpl_scan": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "scpl_scan_stats": (_I, [_P, _P, _I, _I, _I, _P, _P, _P, _P]),
    "scpl_scan_arrivals": (_I, [_P, _P, _I, _I, _I, _P, _I, _P, _P]),
    "scpl_signal_arrival": (_I, [_P, _P, ctypes.c_uint32]),
    "scpl_set_wait_limit": (_I, [_P, ctypes.c_uint64]),
    "scpl_enlarge": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
    "scpl_enlarge_job": (_I, [_P, _P, _I, _I, _I, _I, _I, _I, _P]),
    "scpl_carve_host_many": (_I, [_P, _I, _P, _I, _I, _I, _I, _I, _P, _P]),
    "scpl_blend_sharpness": (_I, [_P, _P, _I, _I, _I, _I, ctypes.POINTER(_LL),
                                  ctypes.POINTER(_LL)]),
    "scpl_seams": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "scpl_carve": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _P]),
    "scpl_carve_host": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _P]),
    "scpl_carve_buffer": (_I, [_P, _P, _I, _I, _I, _P, _I, _I, _P, _P]),
    "scpl_seams_noalloc": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "scpl_copy": (_I, [_P, _P, ctypes.c_size_t, _P]),
    "scpl_isqrt": (_I, [_P, _P, ctypes.c_long, _P]),
    "scpl_set_profiling": (_I, [_P, _I]),
    "scpl_keff_log": (_I, [_P, _P, _I, _P]),
    "scpl_get_stats": (_I, [_P, ctypes.POINTER(Stats)]),
    "scpl_carve_batch": (_I, [_P, ctypes.POINTER(Job), _I]),
    "scpl_tune": (_I, [_P, _I, _I, _I, ctypes.POINTER(Tuning)]),
    "scpl_tuning_set": (_I, [ctypes.POINTER(Tuning)]),
    "scpl_tuning_get": (_I, [_I, _I, ctypes.POINTER(Tuning)]),
    "scpl_tuning_clear": (None, []),
    "scpl_tuning_list": (_I, [ctypes.POINTER(Tuning), _I]),
    "scpl_set_autotune": (_I, [_P, _I]),
    "scpl_server_set_autotune": (_I, [_P, _I]),
    "scpl_job_footprint": (ctypes.c_size_t, [ctypes.POINTER(Params), ctypes.POINTER(Job)]),
    "scpl_job_footprint_per_buffer": (ctypes.c_size_t, [ctypes.POINTER(Job)]),
    "scpl_batch_stats": (_I, [_P, ctypes.POINTER(ServerStats)]),
    "scpl_server_create": (_I, [ctypes.POINTER(Params), ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "scpl_server_submit": (_I, [_P, ctypes.POINTER(Job), ctypes.POINTER(_LL)]),
    "scpl_server_progress": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "scpl_server_poll": (_I, [_P, ctypes.POINTER(_LL), ctypes.POINTER(_I), _I]),
    "scpl_server_drain": (_I, [_P]),
    "scpl_server_cancel": (_I, [_P, _LL]),
    "scpl_server_refuse_allocations": (_I, [_P, _LL, _I]),
    "scpl_server_get_stats": (_I, [_P, ctypes.POINTER(ServerStats)]),
    "scpl_server_last_error": (ctypes.c_char_p, [_P]),
    "scpl_server_destroy": (None, [_P]),
}


class SCPLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libscpl.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def _check(h, status):
    if status != SCPL_OK:
        msg = load().scpl_last_error(h) if h else b""
        raise SCPLError(status, (msg or b"").decode(errors="replace"))


def _dev_ptr(t, dtype, ndim=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype, name="array"):
    if hasattr(a, "numpy"):            # CPU torch tensor
        a = a.numpy()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{name} must be a contiguous {np.dtype(dtype)} array")
    return a.ctypes.data_as(ctypes.c_void_p)


def scpl_default_params() -> Params:
    p = Params()
    load().scpl_default_params(ctypes.byref(p))
    return p


def scpl_create(params: Params | None = None, stream=None):
    """Create a handle on the current CUDA device.  `stream` is a
    torch.cuda.Stream, an integer cudaStream_t, or None (torch's current
    stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    h = ctypes.c_void_p()
    st = load().scpl_create(ctypes.byref(params) if params is not None else None,
                            ctypes.c_void_p(sp), ctypes.byref(h))
    if st != SCPL_OK:
        raise SCPLError(st, "scpl_create failed")
    return h


def scpl_set_stream(h, stream):
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(h, load().scpl_set_stream(h, ctypes.c_void_p(sp)))


def scpl_destroy(h):
    load().scpl_destroy(h)


def scpl_last_error(h) -> str:
    return (load().scpl_last_error(h) or b"").decode(errors="replace")


def scpl_energy(h, frames, energy):
    """frames: cuda uint8 [T,H,W,3]; energy: cuda int32 [T,H,W] (written)."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    T, H, W, _ = frames.shape
    ep = _dev_ptr(energy, torch.int32, 3, "energy")
    if tuple(energy.shape) != (T, H, W):
        raise ValueError("energy must be [T,H,W]")
    _check(h, load().scpl_energy(h, fp, T, H, W, ep))


def scpl_scan(h, frames) -> np.ndarray:
    """Buffer starts (int32, n_buffers + 1 entries, last = T)."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    T, H, W, _ = frames.shape
    starts = np.zeros(T + 1, np.int32)
    nb = ctypes.c_int()
    _check(h, load().scpl_scan(h, fp, T, H, W, starts.ctypes.data_as(_P), ctypes.byref(nb)))
    return starts[: nb.value + 1].copy()


def scpl_scan_stats(h, frames):
    """(buffer starts, A_t int64 [T], emax_t int32 [T]) as the scan computed them."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    T, H, W, _ = frames.shape
    starts = np.zeros(T + 1, np.int32)
    A = np.zeros(T, np.int64)
    M = np.zeros(T, np.int32)
    nb = ctypes.c_int()
    _check(h, load().scpl_scan_stats(h, fp, T, H, W, starts.ctypes.data_as(_P), ctypes.byref(nb),
                                     A.ctypes.data_as(_P), M.ctypes.data_as(_P)))
    return starts[: nb.value + 1].copy(), A, M


def scpl_scan_arrivals(h, frames, arrived, chunk: int) -> np.ndarray:
    """scpl_scan on frames a producer is still copying in: arrived is a cuda
    int32/uint32 tensor of one element, raised (scpl_signal_arrival) to the
    number of complete chunks of `chunk` frames.  Raises SCPLError with
    status SCPL_ETIMEOUT if the counter stops short."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    ap = _counter_ptr(arrived)
    T, H, W, _ = frames.shape
    starts = np.zeros(T + 1, np.int32)
    nb = ctypes.c_int()
    _check(h, load().scpl_scan_arrivals(h, fp, T, H, W, ap, int(chunk),
                                        starts.ctypes.data_as(_P), ctypes.byref(nb)))
    return starts[: nb.value + 1].copy()


def scpl_signal_arrival(stream, counter, value: int):
    """Enqueue on `stream` (a torch.cuda.Stream, a raw handle, or None for
    torch's current stream) the write of `value` to the one-element cuda
    counter tensor."""
    st = load().scpl_signal_arrival(ctypes.c_void_p(_stream_ptr(stream)), _counter_ptr(counter),
                                    int(value))
    if st != SCPL_OK:
        raise SCPLError(st, "scpl_signal_arrival failed")


def scpl_carve_host_many(h, frames: list, target_W: int, k: int, outs: list) -> list[int]:
    """Carve host clips of one shape (numpy uint8 [T,H,W,3], page-locked for
    overlap) into host outputs [T,H,target_W,3], streamed; returns each
    clip's buffer count."""
    n = len(frames)
    if len(outs) != n:
        raise ValueError("one output per clip")
    T, H, W, _ = frames[0].shape
    fps = (ctypes.c_void_p * n)(*[_host_ptr(f, np.uint8, "frames").value for f in frames])
    ops = (ctypes.c_void_p * n)(*[_host_ptr(o, np.uint8, "out").value for o in outs])
    for f, o in zip(frames, outs):
        if f.shape != (T, H, W, 3) or o.shape != (T, H, target_W, 3):
            raise ValueError("clips of one shape, outputs [T,H,target_W,3]")
    nbs = (ctypes.c_int * n)()
    _check(h, load().scpl_carve_host_many(h, n, fps, T, H, W, int(target_W), int(k), ops, nbs))
    return list(nbs)


def scpl_copy(dst, src, stream=None):
    """Copy src into dst (same number of bytes) with the library's host/device
    transfer; each side a torch tensor (CUDA, or CPU page-locked) or a numpy
    array (page-locked).  Asynchronous on `stream` (default: the current
    torch stream)."""
    import torch

    def ptr_bytes(a):
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensors must be contiguous")
            return a.data_ptr(), a.numel() * a.element_size()
        a = np.asarray(a)
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, a.nbytes
    dp, dn = ptr_bytes(dst)
    sp, sn = ptr_bytes(src)
    if dn != sn:
        raise ValueError(f"dst holds {dn} bytes, src {sn}")
    if stream is None:
        stream = torch.cuda.current_stream()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    status = load().scpl_copy(ctypes.c_void_p(dp), ctypes.c_void_p(sp), sn, ctypes.c_void_p(st))
    if status != SCPL_OK:
        raise SCPLError(status, "scpl_copy failed")


def scpl_enlarge(h, frames, target_W: int, k: int, out) -> np.ndarray:
    """Widen cuda uint8 [T,H,W,3] frames to target_W by seam insertion into
    out [T,H,target_W,3]; returns the buffer starts."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    op = _dev_ptr(out, torch.uint8, 4, "out")
    T, H, W, _ = frames.shape
    if tuple(out.shape) != (T, H, target_W, 3):
        raise ValueError("out must be [T,H,target_W,3]")
    starts = np.zeros(T + 1, np.int32)
    nb = ctypes.c_int()
    _check(h, load().scpl_enlarge(h, fp, T, H, W, int(target_W), int(k), op,
                                  starts.ctypes.data_as(_P), ctypes.byref(nb)))
    return starts[: nb.value + 1].copy()


def scpl_enlarge_job(h, frames, target_W: int, target_H: int, k: int, out):
    """Seam insertion along both axes: width first, then the height on the
    transposed clip.  frames [T,H,W,3] uint8 (device), out [T,target_H,target_W,3]."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    op = _dev_ptr(out, torch.uint8, 4, "out")
    T, H, W, _ = frames.shape
    if tuple(out.shape) != (T, target_H, target_W, 3):
        raise ValueError("out must be [T,target_H,target_W,3]")
    _check(h, load().scpl_enlarge_job(h, fp, T, H, W, int(target_W), int(target_H), int(k), op))


def scpl_blend_sharpness(h, frames, window: int = 4) -> tuple[int, int]:
    """(num, den) of the blends of `window` consecutive frames of a cuda
    uint8 [T,H,W,3] clip; num / den is the blends' sharpness (1 = static)."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    T, H, W, _ = frames.shape
    n, d = ctypes.c_longlong(), ctypes.c_longlong()
    _check(h, load().scpl_blend_sharpness(h, fp, T, H, W, int(window), ctypes.byref(n),
                                          ctypes.byref(d)))
    return n.value, d.value


def scpl_isqrt(x, r, stream=None):
    """r = floor(sqrt(x)) by the buffer scan's device routine (Eq. 7-8):
    x cuda int64/uint64 [n] (values below 2^53), r cuda int32/uint32 [n]."""
    import torch
    if x.device.type != "cuda" or r.device.type != "cuda" or x.numel() != r.numel():
        raise ValueError("x and r: CUDA tensors of the same length")
    if x.element_size() != 8 or r.element_size() != 4 or not (x.is_contiguous() and
                                                              r.is_contiguous()):
        raise ValueError("x: contiguous 64-bit, r: contiguous 32-bit")
    if stream is None:
        stream = torch.cuda.current_stream()
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    status = load().scpl_isqrt(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                               x.numel(), ctypes.c_void_p(st))
    if status != SCPL_OK:
        raise SCPLError(status, "scpl_isqrt failed")


def scpl_set_wait_limit(h, ns: int):
    _check(h, load().scpl_set_wait_limit(h, int(ns)))


def _counter_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.numel() == 1
            and t.dtype in (torch.int32, torch.uint32)):
        raise ValueError("counter must be a one-element cuda int32/uint32 tensor")
    return ctypes.c_void_p(t.data_ptr())


def scpl_seams(h, energy, k: int, cols) -> int:
    """energy: cuda int32 [H,W]; cols: cuda int16 [k,H] (written).  Returns k_eff."""
    import torch
    ep = _dev_ptr(energy, torch.int32, 2, "energy")
    H, W = energy.shape
    cp = _dev_ptr(cols, torch.int16, 2, "cols")
    if cols.shape[0] < k or cols.shape[1] != H:
        raise ValueError("cols must be [k,H]")
    ke = ctypes.c_int()
    _check(h, load().scpl_seams(h, ep, H, W, k, cp, ctypes.byref(ke)))
    return ke.value


def scpl_carve(h, frames, target_W: int, k: int, out, seams=None) -> np.ndarray:
    """frames: cuda uint8 [T,H,W,3]; out: cuda uint8 [T,H,target_W,3];
    seams: optional cuda int16 [>=n_buffers, W-target_W, H].  Returns the
    buffer starts."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    T, H, W, _ = frames.shape
    op = _dev_ptr(out, torch.uint8, 4, "out")
    if tuple(out.shape) != (T, H, target_W, 3):
        raise ValueError("out must be [T,H,target_W,3]")
    sp = None
    if seams is not None:
        sp = _dev_ptr(seams, torch.int16, 3, "seams")
        if seams.shape[1] != W - target_W or seams.shape[2] != H:
            raise ValueError("seams must be [n_buffers, W-target_W, H]")
    starts = np.zeros(T + 1, np.int32)
    nb = ctypes.c_int()
    _check(h, load().scpl_carve(h, fp, T, H, W, target_W, k, op, starts.ctypes.data_as(_P),
                                ctypes.byref(nb), sp))
    return starts[: nb.value + 1].copy()


def scpl_carve_buffer(h, frames, target_W: int, k: int, out, prev_frame=None, seams=None):
    """Carve cuda uint8 [T,H,W,3] frames as one fixed buffer into out
    [T,H,target_W,3]; prev_frame (cuda uint8 [H,W,3] or None) is the clip's
    frame before them, for the first frame's motion term.  seams: optional
    cuda int16 [1, W-target_W, H]."""
    import torch
    fp = _dev_ptr(frames, torch.uint8, 4, "frames")
    T, H, W, _ = frames.shape
    op = _dev_ptr(out, torch.uint8, 4, "out")
    if tuple(out.shape) != (T, H, target_W, 3):
        raise ValueError("out must be [T,H,target_W,3]")
    pp = None
    if prev_frame is not None:
        pp = _dev_ptr(prev_frame, torch.uint8, 3, "prev_frame")
        if tuple(prev_frame.shape) != (H, W, 3):
            raise ValueError("prev_frame must be [H,W,3]")
    sp = None
    if seams is not None:
        sp = _dev_ptr(seams, torch.int16, 3, "seams")
        if tuple(seams.shape[1:]) != (W - target_W, H):
            raise ValueError("seams must be [1, W-target_W, H]")
    _check(h, load().scpl_carve_buffer(h, fp, T, H, W, pp, target_W, k, op, sp))


def scpl_carve_host(h, frames, target_W: int, k: int, out, seams=None) -> np.ndarray:
    """Host-memory form: frames uint8 [T,H,W,3], out uint8 [T,H,target_W,3],
    seams optional int16 [T, W-target_W, H] (numpy or CPU tensors)."""
    T, H, W, _ = frames.shape
    fp = _host_ptr(frames, np.uint8, "frames")
    op = _host_ptr(out, np.uint8, "out")
    if tuple(out.shape) != (T, H, target_W, 3):
        raise ValueError("out must be [T,H,target_W,3]")
    sp = None if seams is None else _host_ptr(seams, np.int16, "seams")
    starts = np.zeros(T + 1, np.int32)
    nb = ctypes.c_int()
    _check(h, load().scpl_carve_host(h, fp, T, H, W, target_W, k, op, starts.ctypes.data_as(_P),
                                     ctypes.byref(nb), sp))
    return starts[: nb.value + 1].copy()


def scpl_seams_noalloc(energy, k: int, cols, stream=None) -> int:
    """scpl_seams for callers that may not allocate device memory: works in
    the library's fixed scratch array (H*W <= 2^21, W <= 4096, H <= 65535,
    k <= 64).
    energy: cuda int32 [H,W]; cols: cuda int16 [k,H] (written).  Returns k_eff."""
    import torch
    ep = _dev_ptr(energy, torch.int32, 2, "energy")
    H, W = energy.shape
    cp = _dev_ptr(cols, torch.int16, 2, "cols")
    if cols.shape[0] < k or cols.shape[1] != H:
        raise ValueError("cols must be [k,H]")
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    ke = ctypes.c_int()
    st = load().scpl_seams_noalloc(ep, H, W, k, cp, ctypes.byref(ke), ctypes.c_void_p(sp))
    if st != SCPL_OK:
        raise SCPLError(st, "scpl_seams_noalloc failed (sizes beyond its fixed scratch "
                            "give SCPL_EINVAL)")
    return ke.value


def scpl_keff_log(h) -> list[np.ndarray]:
    """k_eff of every iteration of the last carve, one int32 array per buffer."""
    lib = load()
    n = lib.scpl_keff_log(h, None, 0, None)
    nb = scpl_get_stats(h)["n_buffers"]
    keff = np.zeros(max(n, 1), np.int32)
    iters = np.zeros(max(nb, 1), np.int32)
    lib.scpl_keff_log(h, keff.ctypes.data_as(_P), n, iters.ctypes.data_as(_P))
    out, o = [], 0
    for b in range(nb):
        out.append(keff[o:o + iters[b]].copy())
        o += int(iters[b])
    return out


def scpl_set_profiling(h, on: bool):
    _check(h, load().scpl_set_profiling(h, int(on)))


def scpl_get_stats(h) -> dict:
    """Per-kernel launches, event-timed milliseconds and algorithmic bytes,
    plus the iteration summary of the last carve."""
    st = Stats()
    _check(h, load().scpl_get_stats(h, ctypes.byref(st)))
    kernels = {}
    for i in range(st.n_kernels):
        k = st.kernel[i]
        kernels[k.name.decode()] = {"launches": int(k.launches), "ms": float(k.ms),
                                    "bytes": float(k.bytes)}
    return {"n_buffers": st.n_buffers, "iterations_max": st.iterations_max,
            "iterations_total": int(st.iterations_total), "carved_px": float(st.carved_px),
            "launches": int(st.launches), "kernels": kernels}


class Retargeter:
    """Owns one handle; carve() allocates outputs with torch on the frames'
    device."""

    def __init__(self, alpha: float = 0.20, wg: int = 1, wm: int = 2, t_max: int = 128,
                 use_buffer: bool = True, maxval_mode: int = 0, stream=None, wf: int = 0):
        p = scpl_default_params()
        p.alpha, p.wg, p.wm, p.t_max = alpha, wg, wm, t_max
        p.use_buffer, p.maxval_mode, p.wf = int(use_buffer), maxval_mode, wf
        self.params = p
        self.h = scpl_create(p, stream)

    def carve(self, frames, target_W: int, k: int, with_seams: bool = False):
        import torch
        T, H, W, _ = frames.shape
        out = torch.empty((T, H, target_W, 3), dtype=torch.uint8, device=frames.device)
        seams = None
        if with_seams:
            seams = torch.empty((T, W - target_W, H), dtype=torch.int16, device=frames.device)
        starts = scpl_carve(self.h, frames, target_W, k, out, seams)
        if seams is not None:
            seams = seams[: len(starts) - 1]
        return out, starts, seams

    def enlarge(self, frames, target_W: int, k: int):
        """Widen frames by seam insertion; returns (out, buffer starts)."""
        import torch
        T, H, W, _ = frames.shape
        out = torch.empty((T, H, target_W, 3), dtype=torch.uint8, device=frames.device)
        starts = scpl_enlarge(self.h, frames, target_W, k, out)
        return out, starts

    def enlarge_job(self, frames, target_W: int, target_H: int, k: int):
        """Enlarge frames along both axes by seam insertion; returns out."""
        import torch
        T = frames.shape[0]
        out = torch.empty((T, target_H, target_W, 3), dtype=torch.uint8, device=frames.device)
        scpl_enlarge_job(self.h, frames, target_W, target_H, k, out)
        return out

    def close(self):
        if self.h is not None:
            scpl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batching
def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def make_job(frames, target_W: int, target_H: int, k: int, out, starts=None) -> Job:
    """A Job over torch CUDA tensors (device job) or numpy arrays (host job).
    frames [T,H,W,3] uint8, out [T,target_H,target_W,3] uint8, starts an
    optional int32 numpy array of T+1 entries for the buffer starts."""
    import torch
    j = Job()
    T, H, W, _ = frames.shape
    if isinstance(frames, torch.Tensor):
        j.frames = _dev_ptr(frames, torch.uint8, 4, "frames")
        j.out = _dev_ptr(out, torch.uint8, 4, "out")
        j.on_host = 0
    else:
        j.frames = _host_ptr(frames, np.uint8, "frames")
        j.out = _host_ptr(out, np.uint8, "out")
        j.on_host = 1
    if tuple(out.shape) != (T, target_H, target_W, 3):
        raise ValueError("out must be [T,target_H,target_W,3]")
    j.T, j.H, j.W = T, H, W
    j.target_W, j.target_H, j.k = target_W, target_H, k
    j.buffer_starts = None if starts is None else _host_ptr(starts, np.int32, "starts")
    return j


def _tuning_dict(t: Tuning) -> dict:
    return {"H": t.H, "W": t.W, "dpc_halo": t.dpc_halo, "dpc_warps": t.dpc_warps,
            "dpc_lane_cols": t.dpc_lane_cols, "update_rows": t.update_rows,
            "dp_us": {"r32w4": t.dp_us[0], "r16w4": t.dp_us[1], "r32w8": t.dp_us[2],
                      "r16w8": t.dp_us[3], "single": t.dp_us[4], "r16w4v2": t.dp_us[5],
                      "r16w8v2": t.dp_us[6]},
            "update_us": {1: t.up_us[0], 2: t.up_us[1], 4: t.up_us[2]}}


def scpl_tune(h, H: int, W: int, k: int) -> dict:
    """Measure the kernel choices for (H, W) and record the fastest."""
    t = Tuning()
    _check(h, load().scpl_tune(h, H, W, k, ctypes.byref(t)))
    return _tuning_dict(t)


def scpl_tuning_set(H: int, W: int, dpc_halo: int, update_rows: int, dpc_warps: int = 4,
                    dpc_lane_cols: int = 4):
    t = Tuning()
    t.H, t.W, t.dpc_halo, t.update_rows = H, W, dpc_halo, update_rows
    t.dpc_warps, t.dpc_lane_cols = dpc_warps, dpc_lane_cols
    st = load().scpl_tuning_set(ctypes.byref(t))
    if st != SCPL_OK:
        raise SCPLError(st, "scpl_tuning_set: halo must be 0, 16 or 32, warps 4 or 8, "
                            "columns a lane 4 (or 2 with halo 16) and rows 1, 2 or 4")


def scpl_tuning_get(H: int, W: int) -> dict | None:
    t = Tuning()
    if load().scpl_tuning_get(H, W, ctypes.byref(t)) != SCPL_OK:
        return None
    return _tuning_dict(t)


def scpl_tuning_list() -> list[dict]:
    """Every recorded choice, ordered by (H, W)."""
    n = load().scpl_tuning_list(None, 0)
    arr = (Tuning * max(n, 1))()
    n = min(n, load().scpl_tuning_list(arr, n))
    return [_tuning_dict(arr[i]) for i in range(n)]


def save_tuning(path: str):
    """Write the tuning table to a JSON file (a tuning cache)."""
    import json
    with open(path, "w") as fh:
        json.dump([{k: t[k] for k in ("H", "W", "dpc_halo", "dpc_warps", "dpc_lane_cols",
                                      "update_rows")} for t in scpl_tuning_list()], fh, indent=1)


def load_tuning(path: str) -> int:
    """Restore choices saved by save_tuning; returns how many."""
    import json
    with open(path) as fh:
        entries = json.load(fh)
    for e in entries:
        scpl_tuning_set(e["H"], e["W"], e["dpc_halo"], e["update_rows"], e["dpc_warps"],
                        e["dpc_lane_cols"])
    return len(entries)


def scpl_tuning_clear():
    load().scpl_tuning_clear()


def scpl_set_autotune(h, on: bool):
    _check(h, load().scpl_set_autotune(h, int(on)))


def scpl_job_footprint(params: Params | None, job: Job) -> int:
    return int(load().scpl_job_footprint(ctypes.byref(params) if params is not None else None,
                                         ctypes.byref(job)))


def scpl_job_footprint_per_buffer(job: Job) -> int:
    return int(load().scpl_job_footprint_per_buffer(ctypes.byref(job)))


def scpl_carve_batch(h, jobs: list[Job]) -> list[tuple[int, int]]:
    """Carve every job in one batched run; returns (status, n_buffers) per job
    and raises if any job failed (after all have completed)."""
    arr = (Job * len(jobs))(*jobs)
    st = load().scpl_carve_batch(h, arr, len(jobs))
    res = [(arr[i].status, arr[i].n_buffers) for i in range(len(jobs))]
    _check(h, st)
    return res


def scpl_batch_stats(h) -> dict:
    st = ServerStats()
    _check(h, load().scpl_batch_stats(h, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in ServerStats._fields_}


class Server:
    """Continuous batching of retarget jobs (scpl_server_*).  Tensors and
    arrays of a submitted job are kept referenced here until it completes."""

    def __init__(self, params: Params | None = None, hbm_budget: int = 0, stream=None):
        self.lib = load()
        self.s = ctypes.c_void_p()
        st = self.lib.scpl_server_create(ctypes.byref(params) if params is not None else None,
                                         ctypes.c_size_t(hbm_budget),
                                         ctypes.c_void_p(_stream_ptr(stream)),
                                         ctypes.byref(self.s))
        if st != SCPL_OK:
            raise SCPLError(st, "scpl_server_create failed")
        self._keep: dict[int, tuple] = {}

    def _err(self, st):
        if st != SCPL_OK:
            msg = self.lib.scpl_server_last_error(self.s) or b""
            raise SCPLError(st, msg.decode(errors="replace"))

    def submit(self, frames, target_W: int, target_H: int, k: int, out, starts=None) -> int:
        job = make_job(frames, target_W, target_H, k, out, starts)
        t = ctypes.c_longlong()
        self._err(self.lib.scpl_server_submit(self.s, ctypes.byref(job), ctypes.byref(t)))
        self._keep[t.value] = (frames, out, starts, job)
        return t.value

    def set_autotune(self, on: bool):
        self._err(self.lib.scpl_server_set_autotune(self.s, int(on)))

    def progress(self, wait: bool = False) -> tuple[int, int]:
        a, q = ctypes.c_int(), ctypes.c_int()
        self._err(self.lib.scpl_server_progress(self.s, int(wait), ctypes.byref(a),
                                                ctypes.byref(q)))
        return a.value, q.value

    def poll(self, max_n: int = 1024) -> list[tuple[int, int]]:
        tk = (ctypes.c_longlong * max_n)()
        ss = (ctypes.c_int * max_n)()
        n = self.lib.scpl_server_poll(self.s, tk, ss, max_n)
        done = [(int(tk[i]), int(ss[i])) for i in range(n)]
        for t, _ in done:
            self._keep.pop(t, None)
        return done

    def drain(self):
        self._err(self.lib.scpl_server_drain(self.s))

    def cancel(self, ticket: int):
        """Cancel a job; it completes with SCPL_ECANCELED (reported by poll)."""
        self._err(self.lib.scpl_server_cancel(self.s, int(ticket)))

    def refuse_allocations(self, skip: int, count: int):
        """Fault injection: refuse `count` device allocations after `skip`."""
        self._err(self.lib.scpl_server_refuse_allocations(self.s, int(skip), int(count)))

    def stats(self) -> dict:
        st = ServerStats()
        self._err(self.lib.scpl_server_get_stats(self.s, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.s:
            self.lib.scpl_server_destroy(self.s)
            self.s = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
