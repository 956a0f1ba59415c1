"""Whole-compressor oracle: ST-HOSVD + core quantization + stream (TEST INFRASTRUCTURE ONLY).

Compression (Figure 1 pipeline, restricted to the core):
  1. ST-HOSVD with error control (``oracle.sthosvd``, Algorithm 1, Section 4.1).
  2. Core permuted to the mode storage order (increasing mode size, supplement
     S.2) and vectorised lexicographically (last index fastest).
  3. Quantization target TargetSSE_total - ActualSSE_ST-HOSVD (end of Section
     4.1.3), bit-plane truncation and block encoding (``oracle.quant``).
Factors are stored as raw float64 (factor quantization is not part of this
path).

  4. Core slices left without a significant coefficient (Section 3.3, the
     paragraph after Table 2): after bit-plane truncation such a slice is all
     zero in the decoded core, so the matching factor column is not stored.
     A coefficient is significant when one of its encoded bits is a 1: a 1
     above the last plane p_star, or its leading 1 on p_star where that
     plane's leading bits are encoded (positions <= i_lead).

Full stream layout ("ATC1", little-endian):
  char[4] "ATC1" | u32 version=2 | u32 ndim | u32 dtype (1 f32, 2 f64) |
  u64 dims[ndim] | u64 ranks[ndim] | u32 perm[ndim] | u32 pad to 8 bytes |
  f64 norm2 | f64 sse_trunc |
  u8 kept[mode 0..d-1][ceil(r_i / 8)] (bit c % 8 of byte c / 8: column c of
  U_i stored) | zero pad to 8 bytes |
  f64 factors (mode 0..d-1: n_i x kept_i row-major, the kept columns in
  increasing order) | u64 core_bytes | ATCQ core section
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


def significant(q, p_star, i_lead):
    """Significance of each vectorised coefficient after bit-plane truncation
    (Section 3.3): one of its encoded bits is a 1 -- a 1 above plane p_star, or
    its leading 1 on plane p_star where the leading bits are encoded (positions
    <= i_lead; Supplement S.3 splits the last plane's breakpoint by category)."""
    q = np.asarray(q, dtype=np.uint64)
    n = q.size
    sig = np.zeros(n, dtype=bool)
    if p_star >= 64:
        return sig
    if p_star < 63:
        sig |= (q >> np.uint64(p_star + 1)) != 0
    j = np.arange(n)
    sig |= ((q >> np.uint64(p_star)) != 0) & (j <= i_lead)
    return sig


def kept_columns(sig_vec, ranks, perm):
    """kept[i][c]: slice c of mode i holds a significant coefficient (its factor
    column is stored)."""
    sig = devectorize_core(sig_vec.astype(np.float64), ranks, perm) != 0
    d = len(ranks)
    return [sig.any(axis=tuple(a for a in range(d) if a != i)) for i in range(d)]


def pack_kept(kept):
    out = b""
    for k in kept:
        out += np.packbits(np.asarray(k, dtype=np.uint8), bitorder="little").tobytes()
    if len(out) % 8:
        out += b"\0" * (8 - len(out) % 8)
    return out


def compress(x, rel_eps, rtmss=0.5, mode_order=None, block_size=4096, rank_rule="static"):
    x = np.asarray(x)
    res = sthosvd(x, rel_eps, rtmss=rtmss, mode_order=mode_order, rank_rule=rank_rule)
    ranks = res["ranks"]
    perm = storage_order(ranks)
    vec = vectorize_core(res["core"], perm)
    target_q = res["target_sse"] - res["sse_trunc"]
    core_stream, qinfo = quant.compress_core(vec, target_q, block_size)
    q, _ = quant.quantize(vec, qinfo["k"])
    kept = kept_columns(significant(q, qinfo["p_star"], qinfo["i_lead"]), ranks, perm)
    d = x.ndim
    hdr = b"ATC1" + struct.pack("<III", 2, d, DTYPE_CODE[np.dtype(x.dtype)])
    hdr += struct.pack(f"<{d}Q", *x.shape) + struct.pack(f"<{d}Q", *ranks) + struct.pack(f"<{d}I", *perm)
    if len(hdr) % 8:
        hdr += b"\0" * (8 - len(hdr) % 8)
    hdr += struct.pack("<dd", res["norm2"], res["sse_trunc"])
    hdr += pack_kept(kept)
    body = b"".join(np.ascontiguousarray(u[:, k], dtype="<f8").tobytes() for u, k in zip(res["factors"], kept))
    stream = hdr + body + struct.pack("<Q", len(core_stream)) + core_stream
    info = dict(res)
    info.update(qinfo)
    info.update(perm=perm, target_quant=target_q, core_vec=vec, core_stream=core_stream, kept=kept)
    return stream, info


def parse(stream: bytes):
    if stream[:4] != b"ATC1":
        raise ValueError("bad magic")
    ver, d, dt = struct.unpack_from("<III", stream, 4)
    if ver != 2 or not (1 <= d <= 8) or dt not in CODE_DTYPE:
        raise ValueError("bad header")
    off = 16
    dims = list(struct.unpack_from(f"<{d}Q", stream, off)); off += 8 * d
    ranks = list(struct.unpack_from(f"<{d}Q", stream, off)); off += 8 * d
    perm = list(struct.unpack_from(f"<{d}I", stream, off)); off += 4 * d
    off += (-off) % 8
    norm2, sse_trunc = struct.unpack_from("<dd", stream, off); off += 16
    kept = []
    for i in range(d):
        nb = (ranks[i] + 7) // 8
        bits = np.unpackbits(np.frombuffer(stream, np.uint8, nb, off), bitorder="little")[: ranks[i]]
        kept.append(bits.astype(bool))
        off += nb
    off += (-off) % 8
    factors = []
    for i in range(d):
        nk = int(kept[i].sum())
        cnt = dims[i] * nk
        u = np.zeros((dims[i], ranks[i]))
        u[:, kept[i]] = np.frombuffer(stream, "<f8", cnt, off).reshape(dims[i], nk)
        factors.append(u)
        off += 8 * cnt
    (cb,) = struct.unpack_from("<Q", stream, off); off += 8
    core_stream = stream[off:off + cb]
    return dict(dims=dims, ranks=ranks, perm=perm, dtype=CODE_DTYPE[dt], norm2=norm2,
                sse_trunc=sse_trunc, factors=factors, kept=kept, core_stream=core_stream)


def decompress(stream: bytes):
    h = parse(stream)
    _, _, vec = quant.decode(h["core_stream"])
    core = devectorize_core(vec, h["ranks"], h["perm"])
    order = decompression_order(h["dims"], h["ranks"])
    return reconstruct(core, h["factors"], order)   # float64; cast to h["dtype"] if needed
