"""ctypes front of the C quantizer / encoder oracle (TEST INFRASTRUCTURE ONLY).

Follows Section 3.3 (scaling, rounding, bit planes, breakpoint, leading /
trailing / sign bits), Section 4.2 (independent blocks + size table), Section
4.3 (reconstruction a~ + 2^(p-1), used by the tracker too) and supplement S.6
(rANS of the run lengths).  See ``quant.c`` for the stream layout.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build_oracle

_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_oracle())
        i64, i32 = C.c_int64, C.c_int
        vp = C.c_void_p
        lib.orc_scale_exponent.argtypes = [vp, i64, C.POINTER(i32)]
        lib.orc_quantize.argtypes = [vp, i64, i32, vp, vp]
        lib.orc_quantize.restype = None
        lib.orc_breakpoint.argtypes = [vp, i64, C.c_double, i32, C.POINTER(i32), C.POINTER(i64), vp]
        lib.orc_encode.argtypes = [vp, vp, i64, i32, i32, i64, i32, vp, i64, vp]
        lib.orc_encode.restype = i64
        lib.orc_peek.argtypes = [vp, i64, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)]
        lib.orc_decode.argtypes = [vp, i64, vp, vp, vp, i64]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def scale_exponent(b) -> int:
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    k = C.c_int(0)
    if _L().orc_scale_exponent(_p(b), b.size, C.byref(k)) != 0:
        raise ValueError("core contains NaN or Inf")
    return k.value


def quantize(b, k: int):
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    q = np.empty(b.size, np.uint64)
    s = np.empty(b.size, np.uint8)
    _L().orc_quantize(_p(b), b.size, int(k), _p(q), _p(s))
    return q, s


def breakpoint(q, target: float, k: int):
    """(p_star, i_star, tracked_error_int) -- first position whose tracked
    error (integer units of 2^-2k) is <= target * 2^(2k)."""
    q = np.ascontiguousarray(q, dtype=np.uint64)
    ps, ist = C.c_int(0), C.c_int64(0)
    err = np.zeros(3, np.uint64)
    _L().orc_breakpoint(_p(q), q.size, float(target), int(k), C.byref(ps), C.byref(ist), _p(err))
    e = int(err[0]) | (int(err[1]) << 64) | (int(err[2]) << 128)
    return ps.value, ist.value, e


def encode(q, s, k: int, p_star: int, i_star: int, block_size: int = 4096, categories: bool = False):
    q = np.ascontiguousarray(q, dtype=np.uint64)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    n = q.size
    cat = np.full(n * 64, ord("."), np.uint8) if categories else None
    cap = 1 << 16
    while True:
        out = np.empty(cap, np.uint8)
        r = _L().orc_encode(_p(q), _p(s), n, int(k), int(p_star), int(i_star), int(block_size),
                            _p(out), cap, _p(cat) if cat is not None else None)
        if r == -1:
            raise ValueError("bad arguments to the encoder")
        if r < 0:
            cap = -r
            if cat is not None:
                cat[:] = ord(".")
            continue
        data = out[:r].tobytes()
        if categories:
            return data, cat.reshape(n, 64).view("S1")
        return data


def peek(stream: bytes):
    buf = np.frombuffer(stream, np.uint8)
    n, k, bs, ps, ist = C.c_int64(), C.c_int(), C.c_int(), C.c_int(), C.c_int64()
    if _L().orc_peek(_p(buf), buf.size, C.byref(n), C.byref(k), C.byref(bs), C.byref(ps), C.byref(ist)):
        raise ValueError("not an ATCQ section")
    return dict(n=n.value, k=k.value, block_size=bs.value, p_star=ps.value, i_star=ist.value)


def decode(stream: bytes):
    """Returns (q_tilde, signs, dequantized float64 vector)."""
    buf = np.frombuffer(stream, np.uint8)
    n = peek(stream)["n"]
    qt = np.empty(n, np.uint64)
    sg = np.empty(n, np.uint8)
    b = np.empty(n, np.float64)
    r = _L().orc_decode(_p(buf), buf.size, _p(qt), _p(sg), _p(b), n)
    if r != 0:
        raise ValueError(f"corrupt ATCQ section (code {r})")
    return qt, sg, b


def compress_core(b, target_sse: float, block_size: int = 4096):
    """Vectorised core -> (stream bytes, info).  target_sse in core units."""
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    k = scale_exponent(b)
    q, s = quantize(b, k)
    ps, ist, err = breakpoint(q, target_sse, k)
    data = encode(q, s, k, ps, ist, block_size)
    return data, dict(k=k, p_star=ps, i_star=ist, err_int=err,
                      sse_quant_pred=float(err) * 2.0 ** (-2 * k))
