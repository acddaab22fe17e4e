"""CPU oracle for integer-pel block matching (FSBM and ACBM).

TEST INFRASTRUCTURE ONLY.  The oracle is the independent, slow, plain-C
reference (``me_oracle.c``) that the CUDA library is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package; the library in ``paper_0710_4819_gb300``
never does, and shares no code with it.

The functions here only marshal numpy arrays into the C functions; every step
of the computation is in ``me_oracle.c`` (see its header for the paper
sections each part follows).
"""
from __future__ import annotations

import contextvars
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "me_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libme_oracle.so")
_lock = threading.Lock()
_lib = None
_override = contextvars.ContextVar("oracle_lib", default=None)


class AcbmParams(ctypes.Structure):
    """alpha, beta, gamma = gamma_num/gamma_den, Qp and refinement switch (Sec. 3.2)."""

    _fields_ = [
        ("alpha", ctypes.c_int32),
        ("beta", ctypes.c_int32),
        ("gamma_num", ctypes.c_int32),
        ("gamma_den", ctypes.c_int32),
        ("qp", ctypes.c_int32),
        ("refine", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wextra",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i16p = ctypes.POINTER(ctypes.c_int16)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i32p = ctypes.POINTER(ctypes.c_int32)
    c_int, c_u32 = ctypes.c_int, ctypes.c_uint32
    lib.oracle_lambda_q8.argtypes = [c_int]
    lib.oracle_lambda_q8.restype = c_u32
    lib.oracle_mv_bits.argtypes = [c_int]
    lib.oracle_mv_bits.restype = c_int
    lib.oracle_intra_sad.argtypes = [u8p, c_int, c_int, c_int, c_int, u32p]
    lib.oracle_intra_sad.restype = c_int
    lib.oracle_fsbm.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_u32,
                                i16p, u32p, u32p, c_int]
    lib.oracle_fsbm.restype = c_int
    lib.oracle_fsbm_blocks.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_u32,
                                       i32p, c_int, i16p, u32p, u32p, c_int]
    lib.oracle_fsbm_blocks.restype = c_int
    prm_p = ctypes.POINTER(AcbmParams)
    lib.oracle_acbm.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_u32,
                                i16p, prm_p, i16p, u32p, u8p, u32p, u32p]
    lib.oracle_acbm.restype = c_int
    lib.oracle_acbm_blocks.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_u32,
                                       i16p, i16p, prm_p, i32p, c_int, i16p, u32p, u8p,
                                       u32p, u32p]
    lib.oracle_acbm_blocks.restype = c_int
    lib.oracle_halfpel.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_u32,
                                   i16p, i16p, u32p, u32p]
    lib.oracle_halfpel.restype = c_int
    lib.oracle_sad_deviation.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, u32p, u32p]
    lib.oracle_sad_deviation.restype = c_int
    lib.oracle_sad_deviation_blocks.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int,
                                                ctypes.POINTER(c_int), c_int, u32p, u32p]
    lib.oracle_sad_deviation_blocks.restype = c_int
    lib.oracle_fsbm_pred.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_u32, i16p,
                                     u32p, u32p]
    lib.oracle_fsbm_pred.restype = c_int
    lib.oracle_fsbm_pred_blocks.argtypes = [u8p, u8p, c_int, c_int, c_int, c_int, c_int, c_u32,
                                            i16p, ctypes.POINTER(ctypes.c_int32), c_int, i16p, u32p,
                                            u32p]
    lib.oracle_fsbm_pred_blocks.restype = c_int
    lib.oracle_median_predictor.argtypes = [i16p, c_int, c_int, c_int, ctypes.POINTER(c_int),
                                            ctypes.POINTER(c_int)]
    lib.oracle_median_predictor.restype = None
    return lib


def _load():
    global _lib
    ov = _override.get()
    if ov is not None:
        return ov
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def compile_variant(src_text: str, out_path: str) -> str:
    """Compiles C source text with the oracle's flags into out_path (for tests
    that check the pins against deliberately broken copies of the oracle)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-w", "-o", out_path,
                    c_path], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


class Variant:
    """The oracle's Python interface bound to another compiled copy."""

    def __init__(self, so_path: str):
        self._lib = _bind(ctypes.CDLL(so_path))

    def __getattr__(self, name):
        fn = globals()[name]
        if not callable(fn) or name.startswith("_") or isinstance(fn, type):
            return fn

        def call(*a, **k):
            token = _override.set(self._lib)
            try:
                return fn(*a, **k)
            finally:
                _override.reset(token)
        return call


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray | None, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _frame(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("frames are 2-D uint8 arrays [H, W]")
    return a


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what} returned status {st}")


def lambda_q8(qp: int) -> int:
    return int(_load().oracle_lambda_q8(int(qp)))


def mv_bits(v: int) -> int:
    return int(_load().oracle_mv_bits(int(v)))


def intra_sad(cur, N: int, M: int) -> np.ndarray:
    """Scaled Intra_SAD (NM * Intra_SAD) per block, shape [BH, BW] uint32."""
    cur = _frame(cur)
    H, W = cur.shape
    out = np.zeros((max(H // M, 1), max(W // N, 1)), np.uint32)
    _check(_load().oracle_intra_sad(_ptr(cur, ctypes.c_uint8), W, H, N, M,
                                    _ptr(out, ctypes.c_uint32)), "oracle_intra_sad")
    return out


def fsbm(cur, ref, N: int, M: int, p: int, lam_q8: int, nthreads: int = 1):
    """Full search.  Returns (mv [BH,BW,2] int16, J [BH,BW] u32, sad [BH,BW] u32)."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    if ref.shape != cur.shape:
        raise ValueError("cur and ref differ in shape")
    BH, BW = max(H // M, 1), max(W // N, 1)
    mv = np.zeros((BH, BW, 2), np.int16)
    J = np.zeros((BH, BW), np.uint32)
    sad = np.zeros((BH, BW), np.uint32)
    _check(_load().oracle_fsbm(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W, H, N, M,
                               p, lam_q8, _ptr(mv, ctypes.c_int16), _ptr(J, ctypes.c_uint32),
                               _ptr(sad, ctypes.c_uint32), nthreads), "oracle_fsbm")
    return mv, J, sad


def halfpel(cur, ref, N: int, M: int, p: int, lam_q8: int, mv_int):
    """Half-pel refinement of an integer vector field (Sec. 2.2 / 2.3).
    Returns (mv [BH,BW,2] int16 in half-pel units, J [BH,BW] u32, sad [BH,BW] u32)."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    if ref.shape != cur.shape:
        raise ValueError("cur and ref differ in shape")
    BH, BW = max(H // M, 1), max(W // N, 1)
    mv_int = np.ascontiguousarray(mv_int, dtype=np.int16).reshape(BH, BW, 2)
    mv = np.zeros((BH, BW, 2), np.int16)
    J = np.zeros((BH, BW), np.uint32)
    sad = np.zeros((BH, BW), np.uint32)
    _check(_load().oracle_halfpel(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W, H, N,
                                  M, p, lam_q8, _ptr(mv_int, ctypes.c_int16),
                                  _ptr(mv, ctypes.c_int16), _ptr(J, ctypes.c_uint32),
                                  _ptr(sad, ctypes.c_uint32)), "oracle_halfpel")
    return mv, J, sad


def sad_deviation(cur, ref, N: int, M: int, p: int):
    """SAD_min and SAD_deviation of every block (Sec. 3.1), each [BH,BW] u32."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    if ref.shape != cur.shape:
        raise ValueError("cur and ref differ in shape")
    BH, BW = max(H // M, 1), max(W // N, 1)
    mn = np.zeros((BH, BW), np.uint32)
    dev = np.zeros((BH, BW), np.uint32)
    _check(_load().oracle_sad_deviation(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W, H,
                                        N, M, p, _ptr(mn, ctypes.c_uint32),
                                        _ptr(dev, ctypes.c_uint32)), "oracle_sad_deviation")
    return mn, dev


def fsbm_pred(cur, ref, N: int, M: int, p: int, lam_q8: int):
    """FSBM with R coded against the median predictor of the left, upper and
    upper-right final vectors.  Returns (mv [BH,BW,2] int16, J, sad [BH,BW] u32)."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    if ref.shape != cur.shape:
        raise ValueError("cur and ref differ in shape")
    BH, BW = max(H // M, 1), max(W // N, 1)
    mv = np.zeros((BH, BW, 2), np.int16)
    J = np.zeros((BH, BW), np.uint32)
    sad = np.zeros((BH, BW), np.uint32)
    _check(_load().oracle_fsbm_pred(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W, H, N,
                                    M, p, lam_q8, _ptr(mv, ctypes.c_int16), _ptr(J, ctypes.c_uint32),
                                    _ptr(sad, ctypes.c_uint32)), "oracle_fsbm_pred")
    return mv, J, sad


def fsbm_pred_blocks(cur, ref, N: int, M: int, p: int, lam_q8: int, field, blocks):
    """The listed blocks of the predicted-rate FSBM, each with its predictor
    from `field` [BH,BW,2].  Returns (mv [n,2], J [n], sad [n])."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    field = np.ascontiguousarray(field, dtype=np.int16)
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    mv = np.zeros((len(blocks), 2), np.int16)
    J = np.zeros(len(blocks), np.uint32)
    sad = np.zeros(len(blocks), np.uint32)
    _check(_load().oracle_fsbm_pred_blocks(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W,
                                           H, N, M, p, lam_q8, _ptr(field, ctypes.c_int16),
                                           _ptr(blocks, ctypes.c_int32), len(blocks),
                                           _ptr(mv, ctypes.c_int16), _ptr(J, ctypes.c_uint32),
                                           _ptr(sad, ctypes.c_uint32)), "oracle_fsbm_pred_blocks")
    return mv, J, sad


def median_predictor(mv, bx: int, by: int):
    """The median predictor (pmx, pmy) of block (bx, by) from a field mv [BH,BW,2]."""
    mv = np.ascontiguousarray(mv, dtype=np.int16)
    px, py = ctypes.c_int(0), ctypes.c_int(0)
    _load().oracle_median_predictor(_ptr(mv, ctypes.c_int16), mv.shape[1], bx, by,
                                    ctypes.byref(px), ctypes.byref(py))
    return px.value, py.value


def sad_deviation_blocks(cur, ref, N: int, M: int, p: int, blocks):
    """SAD_min and SAD_deviation of the listed blocks (raster indices), each [n] u32."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    mn = np.zeros(len(blocks), np.uint32)
    dev = np.zeros(len(blocks), np.uint32)
    _check(_load().oracle_sad_deviation_blocks(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8),
                                               W, H, N, M, p, _ptr(blocks, ctypes.c_int),
                                               len(blocks), _ptr(mn, ctypes.c_uint32),
                                               _ptr(dev, ctypes.c_uint32)),
           "oracle_sad_deviation_blocks")
    return mn, dev


def fsbm_blocks(cur, ref, N: int, M: int, p: int, lam_q8: int, blocks, nthreads: int = 1):
    """Full search for the listed block indices (by*BW+bx). Returns (mv [k,2], J [k], sad [k])."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    k = blocks.size
    mv = np.zeros((k, 2), np.int16)
    J = np.zeros(k, np.uint32)
    sad = np.zeros(k, np.uint32)
    _check(_load().oracle_fsbm_blocks(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W, H,
                                      N, M, p, lam_q8, _ptr(blocks, ctypes.c_int32), k,
                                      _ptr(mv, ctypes.c_int16), _ptr(J, ctypes.c_uint32),
                                      _ptr(sad, ctypes.c_uint32), nthreads),
           "oracle_fsbm_blocks")
    return mv, J, sad


def params(alpha=1000, beta=8, gamma_num=1, gamma_den=4, qp=28, refine=1) -> AcbmParams:
    """The paper's defaults alpha=1000, beta=8, gamma=1/4 (Sec. 4)."""
    return AcbmParams(int(alpha), int(beta), int(gamma_num), int(gamma_den), int(qp), int(refine))


def acbm(cur, ref, N: int, M: int, p: int, lam_q8: int, prm: AcbmParams, prev_mv=None):
    """ACBM over a frame.  Returns (mv, J, mask, sad, load), block-grid shaped."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    BH, BW = max(H // M, 1), max(W // N, 1)
    if prev_mv is not None:
        prev_mv = np.ascontiguousarray(prev_mv, dtype=np.int16)
        if prev_mv.shape != (BH, BW, 2):
            raise ValueError("prev_mv must be [BH, BW, 2] int16")
    mv = np.zeros((BH, BW, 2), np.int16)
    J = np.zeros((BH, BW), np.uint32)
    mask = np.zeros((BH, BW), np.uint8)
    sad = np.zeros((BH, BW), np.uint32)
    load = np.zeros((BH, BW), np.uint32)
    _check(_load().oracle_acbm(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W, H, N, M, p,
                               lam_q8, _ptr(prev_mv, ctypes.c_int16), ctypes.byref(prm),
                               _ptr(mv, ctypes.c_int16), _ptr(J, ctypes.c_uint32),
                               _ptr(mask, ctypes.c_uint8), _ptr(sad, ctypes.c_uint32),
                               _ptr(load, ctypes.c_uint32)), "oracle_acbm")
    return mv, J, mask, sad, load


def acbm_blocks(cur, ref, N: int, M: int, p: int, lam_q8: int, prm: AcbmParams, cur_field,
                blocks, prev_mv=None):
    """ACBM for the listed blocks, with spatial predictors read from cur_field."""
    cur, ref = _frame(cur), _frame(ref)
    H, W = cur.shape
    BH, BW = max(H // M, 1), max(W // N, 1)
    cur_field = np.ascontiguousarray(cur_field, dtype=np.int16)
    if cur_field.shape != (BH, BW, 2):
        raise ValueError("cur_field must be [BH, BW, 2] int16")
    if prev_mv is not None:
        prev_mv = np.ascontiguousarray(prev_mv, dtype=np.int16)
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    k = blocks.size
    mv = np.zeros((k, 2), np.int16)
    J = np.zeros(k, np.uint32)
    mask = np.zeros(k, np.uint8)
    sad = np.zeros(k, np.uint32)
    load = np.zeros(k, np.uint32)
    _check(_load().oracle_acbm_blocks(_ptr(cur, ctypes.c_uint8), _ptr(ref, ctypes.c_uint8), W, H,
                                      N, M, p, lam_q8, _ptr(prev_mv, ctypes.c_int16),
                                      _ptr(cur_field, ctypes.c_int16), ctypes.byref(prm),
                                      _ptr(blocks, ctypes.c_int32), k, _ptr(mv, ctypes.c_int16),
                                      _ptr(J, ctypes.c_uint32), _ptr(mask, ctypes.c_uint8),
                                      _ptr(sad, ctypes.c_uint32), _ptr(load, ctypes.c_uint32)),
           "oracle_acbm_blocks")
    return mv, J, mask, sad, load
