"""Pins of the oracle's all-zero-slice factor-column dropping (Section 3.3, the
paragraph after Table 2): after bit-plane truncation a core slice whose
coefficients are all insignificant is zero in the decoded core, so the matching
factor column is not stored.

* significance against a literal bit-by-bit walk of each coefficient's encoded
  bits (planes 63 down to p_star, the last plane's leading bits up to i_lead
  and trailing bits up to i_trail);
* the kept-column maps against brute force over the devectorised core;
* a hand-built core whose last slices are negligible: those columns are
  dropped and the stream is shorter by exactly 8 n_i bytes per dropped column;
* dropping changes nothing in the reconstruction: the same stream with every
  column stored decodes to a bitwise identical tensor (the dropped slices are
  exactly zero, so their columns only add exact zeros).
"""
import struct

import numpy as np

import synth
from oracle import pipeline as P
from oracle import quant as Q
from oracle import sthosvd as O


def _bit_walk_significant(q, p_star, i_lead, i_trail):
    """Walk each coefficient's encoded bits from plane 63 down: planes above
    p_star all, plane p_star as a leading bit (not yet significant) where
    j <= i_lead, as a trailing bit where j <= i_trail; significant = a 1 seen."""
    out = []
    for j, v in enumerate(int(x) for x in q):
        sig = False
        for p in range(63, p_star - 1, -1):
            if p == p_star and not ((sig and j <= i_trail) or (not sig and j <= i_lead)):
                break
            if (v >> p) & 1:
                sig = True
        out.append(sig)
    return np.array(out, dtype=bool)


def test_significance_matches_bit_walk():
    rng = np.random.default_rng(3)
    for trial in range(30):
        n = int(rng.integers(1, 400))
        b = rng.standard_normal(n) * np.exp(-np.arange(n) / max(1.0, n / float(rng.integers(1, 20))))
        frac = float(10 ** rng.uniform(-9, 0.5))
        _, info = Q.compress_core(b, frac * float(np.dot(b, b)), 64)
        q, _ = Q.quantize(b, info["k"])
        got = P.significant(q, info["p_star"], info["i_lead"])
        ref = _bit_walk_significant(q, info["p_star"], info["i_lead"], info["i_trail"])
        assert np.array_equal(got, ref), trial


def test_kept_maps_brute_force():
    rng = np.random.default_rng(4)
    ranks = [3, 5, 4]
    perm = O.storage_order(ranks)
    sig = rng.random(int(np.prod(ranks))) < 0.05
    kept = P.kept_columns(sig, ranks, perm)
    s3 = P.devectorize_core(sig.astype(float), ranks, perm) != 0
    for i in range(3):
        for c in range(ranks[i]):
            assert kept[i][c] == bool(np.take(s3, c, axis=i).any())


def _stream_with_all_columns(stream):
    """The same compressed tensor written with every factor column stored."""
    h = P.parse(stream)
    d = len(h["dims"])
    off = 16 + 16 * d + 4 * d
    off += (-off) % 8
    off += 16
    head = stream[:off]
    full = P.pack_kept([np.ones(r, dtype=bool) for r in h["ranks"]])
    body = b"".join(np.ascontiguousarray(u, dtype="<f8").tobytes() for u in h["factors"])
    return head + full + body + struct.pack("<Q", len(h["core_stream"])) + h["core_stream"]


def test_negligible_slices_are_dropped_and_reconstruction_unchanged():
    # a tensor of multilinear rank (6, 5, 4) compressed at full rank (RTMSS = 0:
    # the whole error budget goes to the quantizer), so the core carries slices
    # that hold only rounding-level coefficients; bit-plane truncation leaves them
    # insignificant
    x = synth.lowrank_tucker((12, 10, 9), (6, 5, 4), noise=None, seed=9)
    xt = x
    stream, info = P.compress(xt, 1e-2, rtmss=0.0)
    kept = info["kept"]
    dropped = [int((~k).sum()) for k in kept]
    assert sum(dropped) >= 1, dropped
    # brute force over the stream's own decoded core
    h = P.parse(stream)
    _, _, vec = Q.decode(h["core_stream"])
    dec = P.devectorize_core(vec, h["ranks"], h["perm"])
    for i in range(3):
        for c in range(h["ranks"][i]):
            assert bool(h["kept"][i][c]) == bool(np.any(np.take(dec, c, axis=i) != 0))
    full = _stream_with_all_columns(stream)
    assert len(full) - len(stream) == 8 * sum(n * dr for n, dr in zip(h["dims"], dropped)) + \
        (len(P.pack_kept([np.ones(r, bool) for r in h["ranks"]])) - len(P.pack_kept(h["kept"])))
    a = P.decompress(stream)
    b = P.decompress(full)
    assert np.array_equal(a, b)
    assert np.linalg.norm(xt - a) <= 1e-2 * np.linalg.norm(xt)


def test_nothing_dropped_when_every_slice_is_significant():
    x = synth.lowrank_tucker()
    stream, info = P.compress(x, 1e-2)
    assert all(k.all() for k in info["kept"])
    assert np.array_equal(P.decompress(stream), P.decompress(_stream_with_all_columns(stream)))
