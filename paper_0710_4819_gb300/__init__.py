"""GB300 (sm_103a) block-matching motion estimation: FSBM and ACBM.

A thin ctypes binding over the C ABI in ``include/me.h`` (``libme.so``).  The
functions keep the C names (``me_fsbm``, ``me_acbm``, ...) and take torch CUDA
tensors; this module only checks shapes and dtypes, allocates outputs and
passes device pointers and the current CUDA stream.  Every step of the
computation runs in the library's CUDA kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

from . import build as _build

__all__ = [
    "load_library", "MeError", "AcbmParams", "me_lambda_q8", "me_mv_bits",
    "me_acbm_default_params", "me_padded_geometry", "me_pad_ref", "me_intra_sad",
    "me_fsbm", "me_acbm", "me_halfpel", "me_halfpel_sequence", "me_sad_deviation",
    "me_motion_study", "me_fsbm_sequence_status", "me_fsbm_pred", "me_fsbm_pred_sequence", "me_fsbm_pred_status", "me_sad_peak", "me_tune_log", "Batch", "Server", "STATUS",
]

_lock = threading.Lock()
_lib = None

STATUS = {0: "ME_OK", 1: "ME_ERR_ARG", 2: "ME_ERR_SHAPE", 3: "ME_ERR_CUDA",
          4: "ME_ERR_NOMEM", 5: "ME_ERR_TIMEOUT", 6: "ME_ERR_BUSY", 7: "ME_ERR_NOTFOUND"}


class MeError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class AcbmParams(ctypes.Structure):
    """me_acbm_params: alpha, beta, gamma = gamma_num/gamma_den, qp, refine (Sec. 3.2)."""

    _fields_ = [("alpha", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("gamma_num", ctypes.c_int32), ("gamma_den", ctypes.c_int32),
                ("qp", ctypes.c_int32), ("refine", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("cur", ctypes.c_void_p), ("ref", ctypes.c_void_p), ("prev_mv", ctypes.c_void_p),
                ("mv_out", ctypes.c_void_p), ("J_out", ctypes.c_void_p),
                ("mask_out", ctypes.c_void_p), ("sad_out", ctypes.c_void_p),
                ("load_out", ctypes.c_void_p), ("lambda_q8", ctypes.c_uint32),
                ("prm", AcbmParams)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_longlong), ("max_inflight", ctypes.c_int),
                ("mode", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int)]


class ServerResult(ctypes.Structure):
    _fields_ = [("has_result", ctypes.c_int), ("status", ctypes.c_int),
                ("latency_ms", ctypes.c_double), ("mv", ctypes.c_void_p), ("J", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("sad", ctypes.c_void_p), ("load", ctypes.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads libme.so (building it first if asked).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"libme.so missing at {path}; run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, c_int, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32
        sig = {
            "me_status_string": ([c_int], ctypes.c_char_p),
            "me_last_error": ([], ctypes.c_char_p),
            "me_lambda_q8": ([ctypes.c_int32], u32),
            "me_mv_bits": ([ctypes.c_int32], ctypes.c_int32),
            "me_acbm_default_params": ([ctypes.c_int32], AcbmParams),
            "me_padded_geometry": ([c_int, c_int, c_int, ctypes.POINTER(c_int),
                                    ctypes.POINTER(c_int), ctypes.POINTER(c_int)], c_int),
            "me_pad_ref": ([vp, c_int, c_int, c_int, vp, vp], c_int),
            "me_intra_sad": ([vp, c_int, c_int, c_int, c_int, vp, vp], c_int),
            "me_fsbm": ([vp, vp, c_int, c_int, c_int, c_int, c_int, u32, vp, vp, vp, vp], c_int),
            "me_acbm": ([vp, vp, c_int, c_int, c_int, c_int, c_int, u32, vp,
                         ctypes.POINTER(AcbmParams), vp, vp, vp, vp, vp, vp], c_int),
            "me_acbm_noalloc": ([vp, vp, c_int, c_int, c_int, c_int, c_int, u32, vp,
                                 ctypes.POINTER(AcbmParams), vp, vp, vp, vp, vp, vp], c_int),
            "me_fsbm_sequence": ([ctypes.POINTER(vp), c_int, c_int, c_int, c_int, c_int, c_int,
                                  u32, vp, vp, vp, vp], c_int),
            "me_halfpel": ([vp, vp, c_int, c_int, c_int, c_int, c_int, u32, vp, vp, vp, vp, vp],
                           c_int),
            "me_halfpel_sequence": ([ctypes.POINTER(vp), c_int, c_int, c_int, c_int, c_int, c_int,
                                     u32, vp, vp, vp, vp, vp], c_int),
            "me_fsbm_sequence_status": ([vp], c_int),
            "me_fsbm_pred": ([vp, vp, c_int, c_int, c_int, c_int, c_int, u32, vp, vp, vp, vp],
                             c_int),
            "me_fsbm_pred_sequence": ([ctypes.POINTER(vp), c_int, c_int, c_int, c_int, c_int, c_int,
                                       u32, vp, vp, vp, vp], c_int),
            "me_fsbm_pred_status": ([c_int, c_int, c_int, c_int, c_int, c_int, vp], c_int),
            "me_sad_deviation": ([vp, vp, c_int, c_int, c_int, c_int, c_int, u32, vp, vp, vp, vp,
                                  vp], c_int),
            "me_motion_study": ([ctypes.POINTER(vp), c_int, c_int, c_int, c_int, c_int, c_int,
                                 u32, vp, vp, vp, vp, vp, vp, vp], c_int),
            "me_acbm_sequence": ([ctypes.POINTER(vp), c_int, c_int, c_int, c_int, c_int, c_int,
                                  u32, vp, ctypes.POINTER(AcbmParams), vp, vp, vp, vp, vp, vp],
                                 c_int),
            "me_acbm_sequence_status": ([c_int, c_int, c_int, c_int, c_int, c_int, vp], c_int),
            "me_tune_log": ([ctypes.c_char_p, c_int], c_int),
            "me_sad_peak": ([c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), vp], c_int),
            "me_batch_create": ([ctypes.POINTER(vp)], c_int),
            "me_batch_add_stream": ([vp, c_int, c_int, c_int, c_int, c_int,
                                     ctypes.POINTER(c_int)], c_int),
            "me_batch_run": ([vp, c_int, ctypes.POINTER(BatchItem), c_int, vp], c_int),
            "me_batch_sync": ([vp, vp], c_int),
            "me_batch_destroy": ([vp], None),
            "me_batch_set_fault": ([vp, ctypes.c_longlong, c_int, c_int], c_int),
            "me_server_create": ([ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)], c_int),
            "me_server_open_stream": ([vp, c_int, c_int, c_int, ctypes.POINTER(AcbmParams),
                                       ctypes.c_int32, ctypes.POINTER(c_int)], c_int),
            "me_server_submit": ([vp, c_int, vp, ctypes.POINTER(ctypes.c_longlong)], c_int),
            "me_server_poll": ([vp, ctypes.c_longlong, ctypes.POINTER(ServerResult)], c_int),
            "me_server_wait": ([vp, ctypes.c_longlong, c_int, ctypes.POINTER(ServerResult)], c_int),
            "me_server_close_stream": ([vp, c_int], c_int),
            "me_server_stats": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(c_int),
                                 ctypes.POINTER(c_int)], c_int),
            "me_server_destroy": ([vp], None),
            "me_server_diagnostics": ([vp], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(st: int, what: str):
    if st != 0:
        detail = ""
        if st == 3:
            detail = load_library().me_last_error().decode()
        raise MeError(st, what, detail)


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _frame_args(cur, ref):
    torch = _torch()
    for t, nm in ((cur, "cur"), (ref, "ref")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8
                and t.dim() == 2 and t.is_contiguous()):
            raise ValueError(f"{nm} must be a contiguous 2-D uint8 CUDA tensor [H, W]")
    if cur.shape != ref.shape:
        raise ValueError("cur and ref differ in shape")
    H, W = cur.shape
    return int(W), int(H)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def me_lambda_q8(qp: int) -> int:
    return int(load_library().me_lambda_q8(int(qp)))


def me_mv_bits(v: int) -> int:
    return int(load_library().me_mv_bits(int(v)))


def me_acbm_default_params(qp: int) -> AcbmParams:
    return load_library().me_acbm_default_params(int(qp))


def params(alpha=1000, beta=8, gamma_num=1, gamma_den=4, qp=28, refine=1) -> AcbmParams:
    return AcbmParams(int(alpha), int(beta), int(gamma_num), int(gamma_den), int(qp), int(refine))


def me_padded_geometry(W: int, H: int, p: int):
    pitch, rows, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().me_padded_geometry(W, H, p, ctypes.byref(pitch), ctypes.byref(rows),
                                             ctypes.byref(P)), "me_padded_geometry")
    return pitch.value, rows.value, P.value


def me_pad_ref(ref, p: int, out=None, stream=None):
    torch = _torch()
    W, H = _frame_args(ref, ref)
    pitch, rows, _ = me_padded_geometry(W, H, p)
    if out is None:
        out = torch.empty((rows, pitch), dtype=torch.uint8, device=ref.device)
    _check(load_library().me_pad_ref(_ptr(ref), W, H, p, _ptr(out), _stream_ptr(stream)),
           "me_pad_ref")
    return out


def me_intra_sad(cur, N: int, M: int, out=None, stream=None):
    torch = _torch()
    W, H = _frame_args(cur, cur)
    if out is None:
        out = torch.empty((max(H // M, 1), max(W // N, 1)), dtype=torch.int32, device=cur.device)
    _check(load_library().me_intra_sad(_ptr(cur), W, H, N, M, _ptr(out), _stream_ptr(stream)),
           "me_intra_sad")
    return out


@dataclass
class FsbmResult:
    mv: "object"     # int16 [BH, BW, 2]
    J: "object"      # int32 view of uint32 [BH, BW]
    sad: "object"    # int32 view of uint32 [BH, BW]


def _outs(H, W, N, M, device):
    torch = _torch()
    BH, BW = max(H // M, 1), max(W // N, 1)
    mv = torch.empty((BH, BW, 2), dtype=torch.int16, device=device)
    J = torch.empty((BH, BW), dtype=torch.int32, device=device)
    sad = torch.empty((BH, BW), dtype=torch.int32, device=device)
    return mv, J, sad


def me_fsbm(cur, ref, N: int, M: int, p: int, lambda_q8: int, out=None, stream=None) -> FsbmResult:
    """Full search of every block (Sec. 2.3).  Outputs: mv int16 [BH,BW,2],
    J and SAD as int32 tensors holding the uint32 values."""
    W, H = _frame_args(cur, ref)
    mv, J, sad = out if out is not None else _outs(H, W, N, M, cur.device)
    _check(load_library().me_fsbm(_ptr(cur), _ptr(ref), W, H, N, M, p, int(lambda_q8), _ptr(mv),
                                  _ptr(J), _ptr(sad), _stream_ptr(stream)), "me_fsbm")
    return FsbmResult(mv, J, sad)


@dataclass
class AcbmResult:
    mv: "object"
    J: "object"
    mask: "object"   # uint8 [BH, BW]
    sad: "object"
    load: "object"


def me_acbm(cur, ref, N: int, M: int, p: int, lambda_q8: int, prm: AcbmParams, prev_mv=None,
            out=None, stream=None) -> AcbmResult:
    """ACBM (Sec. 3.2) for one frame pair; prev_mv is the previous output field."""
    torch = _torch()
    W, H = _frame_args(cur, ref)
    if out is None:
        mv, J, sad = _outs(H, W, N, M, cur.device)
        mask = torch.empty(J.shape, dtype=torch.uint8, device=cur.device)
        load = torch.empty(J.shape, dtype=torch.int32, device=cur.device)
    else:
        mv, J, mask, sad, load = out
    if prev_mv is not None and (prev_mv.dtype != torch.int16 or tuple(prev_mv.shape) != tuple(mv.shape)
                                or not prev_mv.is_contiguous()):
        raise ValueError("prev_mv must be a contiguous int16 [BH, BW, 2] CUDA tensor")
    _check(load_library().me_acbm(_ptr(cur), _ptr(ref), W, H, N, M, p, int(lambda_q8),
                                  _ptr(prev_mv), ctypes.byref(prm), _ptr(mv), _ptr(J), _ptr(mask),
                                  _ptr(sad), _ptr(load), _stream_ptr(stream)), "me_acbm")
    return AcbmResult(mv, J, mask, sad, load)


def _frame_ptrs(frames):
    """frames: uint8 CUDA tensor [K+1, H, W] (contiguous) or a list of [H, W] tensors."""
    torch = _torch()
    if isinstance(frames, torch.Tensor):
        if not (frames.is_cuda and frames.dtype == torch.uint8 and frames.dim() == 3):
            raise ValueError("frames must be a uint8 CUDA tensor [K+1, H, W]")
        frames = [frames[i] for i in range(frames.shape[0])]
    for f in frames:
        if not (f.is_cuda and f.dtype == torch.uint8 and f.dim() == 2 and f.is_contiguous()):
            raise ValueError("each frame must be a contiguous uint8 CUDA tensor [H, W]")
    H, W = frames[0].shape
    arr = (ctypes.c_void_p * len(frames))(*[f.data_ptr() for f in frames])
    return arr, len(frames) - 1, int(W), int(H)


def me_fsbm_sequence(frames, N: int, M: int, p: int, lambda_q8: int, out=None, stream=None):
    """FSBM of K consecutive pairs in one launch; outputs [K, BH, BW, ...]."""
    torch = _torch()
    arr, K, W, H = _frame_ptrs(frames)
    dev = frames[0].device
    if out is None:
        BH, BW = H // M, W // N
        out = (torch.empty((K, BH, BW, 2), dtype=torch.int16, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev))
    mv, J, sad = out
    _check(load_library().me_fsbm_sequence(arr, K, W, H, N, M, p, int(lambda_q8), _ptr(mv), _ptr(J),
                                           _ptr(sad), _stream_ptr(stream)), "me_fsbm_sequence")
    return FsbmResult(mv, J, sad)


def me_halfpel(cur, ref, N: int, M: int, p: int, lambda_q8: int, mv_int, out=None,
               stream=None) -> FsbmResult:
    """Half-pel refinement (Sec. 2.2 / 2.3) of an integer field mv_int
    (int16 [BH,BW,2] on the device).  Outputs: mv int16 [BH,BW,2] in half-pel
    units, J and SAD as int32 tensors holding the uint32 values."""
    W, H = _frame_args(cur, ref)
    mv, J, sad = out if out is not None else _outs(H, W, N, M, cur.device)
    _check(load_library().me_halfpel(_ptr(cur), _ptr(ref), W, H, N, M, p, int(lambda_q8),
                                      _ptr(mv_int), _ptr(mv), _ptr(J), _ptr(sad),
                                      _stream_ptr(stream)), "me_halfpel")
    return FsbmResult(mv, J, sad)


def me_halfpel_sequence(frames, N: int, M: int, p: int, lambda_q8: int, mv_int, out=None,
                        stream=None) -> FsbmResult:
    """me_halfpel for K consecutive pairs in one launch; mv_int and the
    outputs are [K, BH, BW, ...]."""
    torch = _torch()
    arr, K, W, H = _frame_ptrs(frames)
    dev = frames[0].device
    if out is None:
        BH, BW = H // M, W // N
        out = (torch.empty((K, BH, BW, 2), dtype=torch.int16, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev))
    mv, J, sad = out
    _check(load_library().me_halfpel_sequence(arr, K, W, H, N, M, p, int(lambda_q8), _ptr(mv_int),
                                              _ptr(mv), _ptr(J), _ptr(sad), _stream_ptr(stream)),
           "me_halfpel_sequence")
    return FsbmResult(mv, J, sad)


def me_fsbm_sequence_status(stream=None) -> int:
    """Waits for the stream; ME_ERR_TIMEOUT (5) if a bounded wait of a
    persistent FSBM sequence run gave up since the last call, else 0."""
    return load_library().me_fsbm_sequence_status(_stream_ptr(stream))


def me_fsbm_pred(cur, ref, N: int, M: int, p: int, lambda_q8: int, out=None,
                 stream=None) -> FsbmResult:
    """FSBM with R coded against the median predictor of the left, upper and
    upper-right final vectors (a wavefront over the blocks)."""
    W, H = _frame_args(cur, ref)
    mv, J, sad = out if out is not None else _outs(H, W, N, M, cur.device)
    _check(load_library().me_fsbm_pred(_ptr(cur), _ptr(ref), W, H, N, M, p, int(lambda_q8),
                                        _ptr(mv), _ptr(J), _ptr(sad), _stream_ptr(stream)),
           "me_fsbm_pred")
    return FsbmResult(mv, J, sad)


def me_fsbm_pred_sequence(frames, N: int, M: int, p: int, lambda_q8: int, out=None,
                          stream=None) -> FsbmResult:
    """me_fsbm_pred of K consecutive pairs in two launches; outputs [K, BH, BW, ...]."""
    torch = _torch()
    arr, K, W, H = _frame_ptrs(frames)
    dev = frames[0].device
    if out is None:
        BH, BW = H // M, W // N
        out = (torch.empty((K, BH, BW, 2), dtype=torch.int16, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev))
    mv, J, sad = out
    _check(load_library().me_fsbm_pred_sequence(arr, K, W, H, N, M, p, int(lambda_q8), _ptr(mv),
                                                _ptr(J), _ptr(sad), _stream_ptr(stream)),
           "me_fsbm_pred_sequence")
    return FsbmResult(mv, J, sad)


def me_fsbm_pred_status(W: int, H: int, N: int, M: int, p: int, K: int = 1, stream=None) -> int:
    """Waits for the stream; the status of the last predicted-rate run of this shape."""
    return load_library().me_fsbm_pred_status(W, H, N, M, p, K, _stream_ptr(stream))


@dataclass
class SadStats:
    mv: "object"       # int16 [..., BH, BW, 2] FSBM vector
    J: "object"        # int32 view of uint32 [..., BH, BW] (None for a study)
    intra: "object"    # int32 view of uint32 [..., BH, BW]: N*M*Intra_SAD (None for one pair)
    sad_min: "object"  # int32 view of uint32 [..., BH, BW]
    sad_dev: "object"  # int32 view of uint32 [..., BH, BW]
    err: "object"      # uint8 [..., BH, BW]: L1 error against the known vector (None for one pair)


def me_sad_deviation(cur, ref, N: int, M: int, p: int, lambda_q8: int = 0, stream=None) -> SadStats:
    """FSBM plus SAD_min and SAD_deviation of every block (Sec. 3.1)."""
    torch = _torch()
    W, H = _frame_args(cur, ref)
    mv, J, smin = _outs(H, W, N, M, cur.device)
    sdev = torch.empty_like(smin)
    _check(load_library().me_sad_deviation(_ptr(cur), _ptr(ref), W, H, N, M, p, int(lambda_q8),
                                            _ptr(mv), _ptr(J), _ptr(smin), _ptr(sdev),
                                            _stream_ptr(stream)), "me_sad_deviation")
    return SadStats(mv, J, None, smin, sdev, None)


def me_motion_study(frames, true_mv, N: int, M: int, p: int, lambda_q8: int = 0,
                    stream=None) -> SadStats:
    """The known-motion experiment of Sec. 3.1 in one launch: frames[0] the
    original, frames[1..K] moved by true_mv (int16 CUDA [K, 2], (gx, gy));
    outputs [K, BH, BW, ...]."""
    torch = _torch()
    arr, K, W, H = _frame_ptrs(frames)
    dev = frames[0].device
    if not (true_mv.is_cuda and true_mv.dtype == torch.int16 and tuple(true_mv.shape) == (K, 2)
            and true_mv.is_contiguous()):
        raise ValueError("true_mv must be a contiguous int16 CUDA tensor [K, 2]")
    BH, BW = H // M, W // N
    mv = torch.empty((K, BH, BW, 2), dtype=torch.int16, device=dev)
    intra, smin, sdev = (torch.empty((K, BH, BW), dtype=torch.int32, device=dev) for _ in range(3))
    err = torch.empty((K, BH, BW), dtype=torch.uint8, device=dev)
    _check(load_library().me_motion_study(arr, K, W, H, N, M, p, int(lambda_q8), _ptr(true_mv),
                                           _ptr(mv), _ptr(intra), _ptr(smin), _ptr(sdev),
                                           _ptr(err), _stream_ptr(stream)), "me_motion_study")
    return SadStats(mv, None, intra, smin, sdev, err)


def me_acbm_sequence(frames, N: int, M: int, p: int, lambda_q8: int, prm: AcbmParams,
                     prev_mv=None, out=None, stream=None) -> AcbmResult:
    """ACBM of K consecutive pairs in one persistent launch (pairs overlap)."""
    torch = _torch()
    arr, K, W, H = _frame_ptrs(frames)
    dev = frames[0].device
    if out is None:
        BH, BW = H // M, W // N
        out = (torch.empty((K, BH, BW, 2), dtype=torch.int16, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev),
               torch.empty((K, BH, BW), dtype=torch.uint8, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev),
               torch.empty((K, BH, BW), dtype=torch.int32, device=dev))
    mv, J, mask, sad, load = out
    _check(load_library().me_acbm_sequence(arr, K, W, H, N, M, p, int(lambda_q8), _ptr(prev_mv),
                                           ctypes.byref(prm), _ptr(mv), _ptr(J), _ptr(mask),
                                           _ptr(sad), _ptr(load), _stream_ptr(stream)),
           "me_acbm_sequence")
    return AcbmResult(mv, J, mask, sad, load)


def me_acbm_sequence_status(W: int, H: int, N: int, M: int, p: int, K: int, stream=None):
    _check(load_library().me_acbm_sequence_status(W, H, N, M, p, K, _stream_ptr(stream)),
           "me_acbm_sequence")


def me_sad_peak(variant: int = 0, stream=None):
    """(absdiff/s, lane-ops per clock per SM) of a packed-SAD instruction form."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().me_sad_peak(variant, ctypes.byref(a), ctypes.byref(b),
                                      _stream_ptr(stream)), "me_sad_peak")
    return a.value, b.value


def me_tune_log() -> str:
    """The autotuner's record: one line per tuned shape (model's and chosen
    candidate, every candidate's best time in ms)."""
    lib = load_library()
    need = lib.me_tune_log(None, 0)
    buf = ctypes.create_string_buffer(max(1, need))
    lib.me_tune_log(buf, need)
    return buf.value.decode()


class Batch:
    """me_batch: many streams of uneven size, one persistent launch per step."""

    def __init__(self):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.me_batch_create(ctypes.byref(h)), "me_batch_create")
        self._h = h
        self.shapes = []

    def add_stream(self, W: int, H: int, N: int, M: int, p: int) -> int:
        idx = ctypes.c_int()
        _check(self._lib.me_batch_add_stream(self._h, W, H, N, M, p, ctypes.byref(idx)),
               "me_batch_add_stream")
        self.shapes.append((W, H, N, M, p))
        return idx.value

    def run(self, mode: int, items, stream=None):
        arr = (BatchItem * len(items))(*items)
        _check(self._lib.me_batch_run(self._h, int(mode), arr, len(items), _stream_ptr(stream)),
               "me_batch_run")

    def set_fault(self, timeout_ns: int, skip_stream: int = -1, skip_block: int = -1):
        _check(self._lib.me_batch_set_fault(self._h, int(timeout_ns), int(skip_stream),
                                            int(skip_block)), "me_batch_set_fault")

    def sync(self, stream=None):
        _check(self._lib.me_batch_sync(self._h, _stream_ptr(stream)), "me_batch_sync")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.me_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """me_server: continuous-batching request server over many streams.

    submit() takes one uint8 numpy frame [H, W] (host memory); results come
    back as numpy arrays from poll()/wait().
    """

    def __init__(self, budget_bytes: int, max_inflight: int = 2, mode: int = 1, N: int = 16,
                 M: int = 16):
        self._lib = load_library()
        self.N, self.M, self.mode = N, M, mode
        cfg = ServerConfig(int(budget_bytes), int(max_inflight), int(mode), int(N), int(M))
        h = ctypes.c_void_p()
        _check(self._lib.me_server_create(ctypes.byref(cfg), ctypes.byref(h)), "me_server_create")
        self._h = h
        self.shapes = {}

    def open_stream(self, W: int, H: int, p: int, qp: int = 28, prm: AcbmParams | None = None) -> int:
        sid = ctypes.c_int()
        _check(self._lib.me_server_open_stream(self._h, W, H, p,
                                               None if prm is None else ctypes.byref(prm),
                                               int(qp), ctypes.byref(sid)), "me_server_open_stream")
        self.shapes[sid.value] = (W, H)
        return sid.value

    def submit(self, stream_id: int, frame) -> int:
        import numpy as np
        W, H = self.shapes[stream_id]
        f = np.ascontiguousarray(frame, dtype=np.uint8)
        if f.shape != (H, W):
            raise ValueError(f"frame must be [{H}, {W}] uint8")
        rid = ctypes.c_longlong()
        _check(self._lib.me_server_submit(self._h, stream_id, f.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.byref(rid)), "me_server_submit")
        return rid.value

    def _result(self, stream_id):
        import numpy as np
        W, H = self.shapes[stream_id]
        BH, BW = H // self.M, W // self.N
        out = dict(mv=np.zeros((BH, BW, 2), np.int16), J=np.zeros((BH, BW), np.uint32),
                   mask=np.zeros((BH, BW), np.uint8), sad=np.zeros((BH, BW), np.uint32),
                   load=np.zeros((BH, BW), np.uint32))
        res = ServerResult(0, 0, 0.0, *(out[k].ctypes.data_as(ctypes.c_void_p).value
                                        for k in ("mv", "J", "mask", "sad", "load")))
        return res, out

    def poll(self, request_id: int, stream_id: int):
        """None while pending, else (has_result, latency_ms, arrays)."""
        res, out = self._result(stream_id)
        st = self._lib.me_server_poll(self._h, request_id, ctypes.byref(res))
        if st == 6:
            return None
        _check(st, "me_server_poll")
        return bool(res.has_result), res.latency_ms, out

    def wait(self, request_id: int, stream_id: int, timeout_ms: int = 10000):
        res, out = self._result(stream_id)
        st = self._lib.me_server_wait(self._h, request_id, int(timeout_ms), ctypes.byref(res))
        _check(st, "me_server_wait")
        return bool(res.has_result), res.latency_ms, out

    def diagnostics(self) -> str:
        return self._lib.me_server_diagnostics(self._h).decode()

    def close_stream(self, stream_id: int):
        _check(self._lib.me_server_close_stream(self._h, stream_id), "me_server_close_stream")

    def stats(self):
        used, nstr, pend = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        st = self._lib.me_server_stats(self._h, ctypes.byref(used), ctypes.byref(nstr),
                                       ctypes.byref(pend))
        _check(st, "me_server_stats")
        return used.value, nstr.value, pend.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.me_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

