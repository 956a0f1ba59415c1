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
        lib.orc_encode.argtypes = [vp, vp, i64, i32, i32, i32, i64, i64, i32, vp, i64, vp]
        lib.orc_encode.restype = i64
        lib.orc_peek.argtypes = [vp, i64, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                 C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]
        lib.orc_decode.argtypes = [vp, i64, vp, vp, vp, i64]
        lib.orc_plane_rans_bytes.argtypes = [vp, vp, i64, i32, i32]
        lib.orc_plane_rans_bytes.restype = i64
        lib.orc_plane_stats.argtypes = [vp, i64, i32, vp, vp, C.POINTER(i64), C.POINTER(i64)]
        lib.orc_plane_stats.restype = None
        lib.orc_split_walk.argtypes = [vp, i64, i32, i32, C.c_double, i32, C.POINTER(i64), C.POINTER(i64), vp]
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


def _signed192(w):
    v = int(w[0]) | (int(w[1]) << 64) | (int(w[2]) << 128)
    return v - (1 << 192) if v >> 191 else v


def plane_efficiencies(q, s, p: int, block_size: int):
    """Exact encoding statistics of plane p encoded whole (Supplement S.3):
    SSE reduction and bit cost of its leading bits (rANS bytes x 8 + one sign
    bit per leading 1) and of its trailing bits (one raw bit each)."""
    q = np.ascontiguousarray(q, dtype=np.uint64)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    dl = np.zeros(3, np.uint64)
    dt = np.zeros(3, np.uint64)
    ones, trail = C.c_int64(0), C.c_int64(0)
    _L().orc_plane_stats(_p(q), q.size, int(p), _p(dl), _p(dt), C.byref(ones), C.byref(trail))
    rb = _L().orc_plane_rans_bytes(_p(q), _p(s), q.size, int(block_size), int(p))
    if rb < 0:
        raise ValueError("plane cost failed")
    return dict(d_lead=_signed192(dl), d_trail=_signed192(dt), cost_lead=8 * int(rb) + ones.value,
                cost_trail=trail.value)


def split_priority(q, s, p_star: int, block_size: int) -> int:
    """0: leading bits first on plane p_star, 1: trailing bits first.  The
    category with the higher efficiency (SSE reduction / encoding cost) on the
    previous plane p_star + 1 goes first, compared exactly as
    d_lead * cost_trail >= d_trail * cost_lead (ties and empty categories:
    leading first); on the top plane there is no previous plane: leading first."""
    if p_star >= 63:
        return 0
    e = plane_efficiencies(q, s, p_star + 1, block_size)
    return 0 if e["d_lead"] * e["cost_trail"] >= e["d_trail"] * e["cost_lead"] else 1


def split_breakpoint(q, s, target: float, k: int, block_size: int):
    """(p_star, prio, i_lead, i_trail, tracked error): the plane of the
    breakpoint search in coefficient order (Section 3.3), then the split walk
    of that plane in priority order (Supplement S.3).  When the split walk
    does not reach the target on the plane (the coefficient-order walk dipped
    below it only transiently), the plane keeps its single breakpoint."""
    q = np.ascontiguousarray(q, dtype=np.uint64)
    p_star, i_star, err = breakpoint(q, target, k)
    if p_star >= 64:
        return p_star, 0, q.size - 1, q.size - 1, err
    prio = split_priority(q, s, p_star, block_size)
    il, it = C.c_int64(0), C.c_int64(0)
    e = np.zeros(3, np.uint64)
    hit = _L().orc_split_walk(_p(q), q.size, int(p_star), int(prio), float(target), int(k), C.byref(il), C.byref(it), _p(e))
    if not hit:
        return p_star, prio, i_star, i_star, err
    return p_star, prio, il.value, it.value, int(e[0]) | (int(e[1]) << 64) | (int(e[2]) << 128)


def encode(q, s, k: int, p_star: int, i_lead: int, i_trail: int | None = None, block_size: int = 4096,
           categories: bool = False, prio: int = 0):
    """Encode with the breakpoints (i_lead, i_trail) of the last plane; i_trail
    None: the single breakpoint of Section 3.3 (i_trail = i_lead)."""
    if i_trail is None:
        i_trail = i_lead
    q = np.ascontiguousarray(q, dtype=np.uint64)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    n = q.size
    cat = np.full(n * 64, ord("."), np.uint8) if categories else None
    cap = 1 << 16
    while True:
        out = np.empty(cap, np.uint8)
        r = _L().orc_encode(_p(q), _p(s), n, int(k), int(p_star), int(prio), int(i_lead), int(i_trail),
                            int(block_size), _p(out), cap, _p(cat) if cat is not None else None)
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
    n, k, bs, ps, pr, il, it = C.c_int64(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
    if _L().orc_peek(_p(buf), buf.size, C.byref(n), C.byref(k), C.byref(bs), C.byref(ps), C.byref(pr), C.byref(il),
                     C.byref(it)):
        raise ValueError("not an ATCQ section")
    return dict(n=n.value, k=k.value, block_size=bs.value, p_star=ps.value, prio=pr.value, i_lead=il.value,
                i_trail=it.value)


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


def compress_core(b, target_sse: float, block_size: int = 4096, split: bool = True):
    """Vectorised core -> (stream bytes, info).  target_sse in core units.
    split: split bit-plane truncation of the last plane (Supplement S.3);
    False: the single breakpoint of Section 3.3."""
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    k = scale_exponent(b)
    q, s = quantize(b, k)
    if split:
        ps, prio, il, it, err = split_breakpoint(q, s, target_sse, k, block_size)
    else:
        ps, il, err = breakpoint(q, target_sse, k)
        prio, it = 0, il
    data = encode(q, s, k, ps, il, it, block_size, prio=prio)
    return data, dict(k=k, p_star=ps, prio=prio, i_lead=il, i_trail=it, err_int=err,
                      sse_quant_pred=float(err) * 2.0 ** (-2 * k))
