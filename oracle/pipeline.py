"""Whole-compressor oracle: ST-HOSVD + core quantization + stream (TEST INFRASTRUCTURE ONLY).

Compression (Figure 1 pipeline, restricted to the core):
  1. ST-HOSVD with error control (``oracle.sthosvd``, Algorithm 1, Section 4.1).
  2. Core permuted to the mode storage order (increasing mode size, supplement
     S.2) and vectorised lexicographically (last index fastest).
  3. Quantization target TargetSSE_total - ActualSSE_ST-HOSVD (end of Section
     4.1.3), bit-plane truncation and block encoding (``oracle.quant``).
Factors are stored as raw float64 (factor quantization is not part of this
path).

Full stream layout ("ATC1", little-endian):
  char[4] "ATC1" | u32 version=1 | u32 ndim | u32 dtype (1 f32, 2 f64) |
  u64 dims[ndim] | u64 ranks[ndim] | u32 perm[ndim] | u32 pad to 8 bytes |
  f64 norm2 | f64 sse_trunc | f64 factors (mode 0..d-1, n_i x r_i row-major) |
  u64 core_bytes | ATCQ core section
"""
from __future__ import annotations

import struct

import numpy as np

from . import quant
from .sthosvd import decompression_order, reconstruct, sthosvd, storage_order

DTYPE_CODE = {np.dtype(np.float32): 1, np.dtype(np.float64): 2}
CODE_DTYPE = {1: np.float32, 2: np.float64}


def vectorize_core(core, perm):
    return np.ascontiguousarray(np.transpose(core, perm)).ravel()


def devectorize_core(vec, ranks, perm):
    shp = [ranks[p] for p in perm]
    t = np.asarray(vec, dtype=np.float64).reshape(shp)
    inv = np.argsort(perm)
    return np.ascontiguousarray(np.transpose(t, inv))


def compress(x, rel_eps, rtmss=0.5, mode_order=None, block_size=4096, rank_rule="static"):
    x = np.asarray(x)
    res = sthosvd(x, rel_eps, rtmss=rtmss, mode_order=mode_order, rank_rule=rank_rule)
    ranks = res["ranks"]
    perm = storage_order(ranks)
    vec = vectorize_core(res["core"], perm)
    target_q = res["target_sse"] - res["sse_trunc"]
    core_stream, qinfo = quant.compress_core(vec, target_q, block_size)
    d = x.ndim
    hdr = b"ATC1" + struct.pack("<III", 1, d, DTYPE_CODE[np.dtype(x.dtype)])
    hdr += struct.pack(f"<{d}Q", *x.shape) + struct.pack(f"<{d}Q", *ranks) + struct.pack(f"<{d}I", *perm)
    if len(hdr) % 8:
        hdr += b"\0" * (8 - len(hdr) % 8)
    hdr += struct.pack("<dd", res["norm2"], res["sse_trunc"])
    body = b"".join(np.ascontiguousarray(u, dtype="<f8").tobytes() for u in res["factors"])
    stream = hdr + body + struct.pack("<Q", len(core_stream)) + core_stream
    info = dict(res)
    info.update(qinfo)
    info.update(perm=perm, target_quant=target_q, core_vec=vec, core_stream=core_stream)
    return stream, info


def parse(stream: bytes):
    if stream[:4] != b"ATC1":
        raise ValueError("bad magic")
    ver, d, dt = struct.unpack_from("<III", stream, 4)
    if ver != 1 or not (1 <= d <= 8) or dt not in CODE_DTYPE:
        raise ValueError("bad header")
    off = 16
    dims = list(struct.unpack_from(f"<{d}Q", stream, off)); off += 8 * d
    ranks = list(struct.unpack_from(f"<{d}Q", stream, off)); off += 8 * d
    perm = list(struct.unpack_from(f"<{d}I", stream, off)); off += 4 * d
    off += (-off) % 8
    norm2, sse_trunc = struct.unpack_from("<dd", stream, off); off += 16
    factors = []
    for i in range(d):
        cnt = dims[i] * ranks[i]
        factors.append(np.frombuffer(stream, "<f8", cnt, off).reshape(dims[i], ranks[i]).astype(np.float64))
        off += 8 * cnt
    (cb,) = struct.unpack_from("<Q", stream, off); off += 8
    core_stream = stream[off:off + cb]
    return dict(dims=dims, ranks=ranks, perm=perm, dtype=CODE_DTYPE[dt], norm2=norm2,
                sse_trunc=sse_trunc, factors=factors, core_stream=core_stream)


def decompress(stream: bytes):
    h = parse(stream)
    _, _, vec = quant.decode(h["core_stream"])
    core = devectorize_core(vec, h["ranks"], h["perm"])
    order = decompression_order(h["dims"], h["ranks"])
    return reconstruct(core, h["factors"], order)   # float64; cast to h["dtype"] if needed
