"""Pins of the C quantizer / tracker / encoder oracle.

* Table 2 worked example (Section 3.3): bit categories, significant set and
  stored signs for the breakpoint the paper gives.
* A literal bit-by-bit simulator in Python big integers (Section 3.3 with the
  Section 4.3 reconstruction): recomputes the whole error after every bit, so
  the oracle's incremental exact tracking is checked against brute force.
* Section 4.3 expectations: 2^(2p)/12 with the reconstruction offset,
  2^(2p)/3 without it.
* Scaling rule 2^63 <= 2^k max|b| < 2^64 checked in exact integers.
* Round trips through the block encoder / rANS decoder.
"""
from fractions import Fraction
import os

import numpy as np
import pytest

import synth
from oracle import pipeline as P
from oracle import quant as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_bitplanes.txt")


def _load_table2():
    rows, bp = [], None
    for line in open(GOLDEN):
        if line.startswith("# breakpoint:"):
            bp = tuple(int(v) for v in line.split(":")[1].split())
        if not line.strip() or line.startswith("#"):
            continue
        name, sign, bits, cat, sig = line.split()
        rows.append((name, int(sign), bits, cat, int(sig)))
    return rows, bp


def test_table2_categories_significance_and_signs():
    rows, (p_star, i_star) = _load_table2()
    q = np.array([sum(int(c) << (63 - j) for j, c in enumerate(bits)) for _, _, bits, _, _ in rows], np.uint64)
    s = np.array([sg for _, sg, _, _, _ in rows], np.uint8)
    data, cat = Q.encode(q, s, 0, p_star, i_star, block_size=32, categories=True)
    for j, (name, sg, bits, cexp, sig) in enumerate(rows):
        got = b"".join(cat[j, :10]).decode()
        assert got == cexp, (name, got, cexp)
    qt, sg_dec, _ = Q.decode(data)
    significant = [int(v != 0) for v in qt]
    assert significant == [r[4] for r in rows]
    assert [rows[j][0] for j in range(8) if not significant[j]] == ["b112", "b121", "b211"]
    for j, r in enumerate(rows):
        keep = 64 - (p_star if j <= i_star else p_star + 1)
        assert int(qt[j]) == (int(q[j]) >> (64 - keep)) << (64 - keep)
        if significant[j]:
            assert sg_dec[j] == r[1]


def _literal_breakpoint(q, target_int):
    """Bit-by-bit walk; after every bit the whole error is recomputed from the
    decoded state (no incremental bookkeeping)."""
    n = len(q)
    known = [0] * n            # bits decoded so far
    lowest = [64] * n          # lowest decoded plane

    def total():
        e = 0
        for i in range(n):
            if known[i] == 0:
                e += q[i] * q[i]
            else:
                p = lowest[i]
                rec = known[i] + ((1 << (p - 1)) if p >= 1 else 0)
                e += (q[i] - rec) ** 2
        return e

    if target_int is not None and total() <= target_int:
        return 64, n - 1, total()
    for p in range(63, -1, -1):
        for i in range(n):
            known[i] |= q[i] & (1 << p)
            lowest[i] = p
            if target_int is not None and total() <= target_int:
                return p, i, total()
    return 0, n - 1, total()


def _target_int(t, k):
    if t < 0:
        return None
    return int(Fraction(t) * Fraction(2) ** (2 * k) // 1)


def test_breakpoint_matches_literal_bit_by_bit_simulation():
    rng = np.random.default_rng(4)
    for trial in range(60):
        n = int(rng.integers(1, 13))
        b = rng.standard_normal(n) * np.exp(-rng.uniform(0, 8, n))
        if trial % 7 == 0:
            b[: max(1, n // 2)] = 0.0
        k = Q.scale_exponent(b)
        q, s = Q.quantize(b, k)
        nb = float(np.dot(b, b))
        for frac in (1.0, 0.3, 1e-2, 1e-5, 1e-9, 0.0, -1.0):
            t = frac * nb
            ps, ist, err = Q.breakpoint(q, t, k)
            lp, li, lerr = _literal_breakpoint([int(v) for v in q], _target_int(t, k))
            assert (ps, ist, err) == (lp, li, lerr), (trial, frac)


def test_scale_exponent_rule():
    rng = np.random.default_rng(3)
    cases = [rng.standard_normal(20) * 10.0 ** rng.uniform(-30, 30) for _ in range(50)]
    cases += [np.array([1.0]), np.array([-0.5, 0.25]), np.array([2.0 ** 70]), np.array([2.0 ** -900, 0.0])]
    for b in cases:
        k = Q.scale_exponent(b)
        m = Fraction(float(np.max(np.abs(b))))
        scaled = m * Fraction(2) ** k
        assert Fraction(2) ** 63 <= scaled < Fraction(2) ** 64
        q, _ = Q.quantize(b, k)
        for v, qv in zip(b, q):
            exact = Fraction(float(abs(v))) * Fraction(2) ** k
            assert abs(Fraction(int(qv)) - exact) <= Fraction(1, 2)
    assert Q.scale_exponent(np.zeros(4)) == 0


def test_reconstruction_offset_expectations():
    """Section 4.3: a in [a~, a~ + 2^p) uniform -> E[(a - a~ - 2^(p-1))^2] = 2^(2p)/12
    (the oracle's reconstruction) versus 2^(2p)/3 at the lower edge."""
    rng = np.random.default_rng(8)
    p = 20
    n = 40000
    low = rng.integers(0, 1 << p, size=n, dtype=np.uint64)
    top = np.uint64(1) << np.uint64(62)
    q = top | low
    s = np.zeros(n, np.uint8)
    data = Q.encode(q, s, 0, p, n - 1, block_size=4096)
    qt, _, deq = Q.decode(data)
    rec = deq  # k = 0: dequantized values are the integer reconstruction
    a = q.astype(np.float64)
    with_c = np.mean((a - rec) ** 2) / 2.0 ** (2 * p)
    without = np.mean((a - qt.astype(np.float64)) ** 2) / 2.0 ** (2 * p)
    assert abs(with_c - 1 / 12) < 0.004
    assert abs(without - 1 / 3) < 0.01


@pytest.mark.parametrize("n,bs,frac", [(1, 32, 1e-3), (31, 32, 1e-6), (5000, 64, 1e-4),
                                        (70000, 4096, 1e-6), (9000, 128, 0.0), (300, 32, 2.0)])
def test_round_trip_and_predicted_error(n, bs, frac):
    rng = np.random.default_rng(n)
    b = rng.standard_normal(n) * np.exp(-np.arange(n) / max(1, n / 5))
    t = frac * float(np.dot(b, b))
    data, info = Q.compress_core(b, t, bs)
    qt, sg, deq = Q.decode(data)
    k = info["k"]
    q, s = Q.quantize(b, k)
    ps, il, it = info["p_star"], info["i_lead"], info["i_trail"]
    err = 0
    for i in range(n):
        # the lowest encoded plane, from the definition: planes above p_star
        # all; p_star for a significant-above coefficient up to i_trail, for a
        # not-yet-significant one up to i_lead (Section 3.3, Supplement S.3)
        above = ps < 63 and (int(q[i]) >> (ps + 1)) != 0
        p_i = ps if (above and i <= it) or (not above and i <= il) else ps + 1
        keep = 0 if p_i >= 64 else (int(q[i]) >> p_i) << p_i
        assert int(qt[i]) == keep
        if keep:
            rec = keep + ((1 << (p_i - 1)) if p_i >= 1 else 0)
            assert sg[i] == s[i]
            assert deq[i] == (-1.0 if s[i] else 1.0) * np.ldexp(float(rec), -k)
        else:
            rec = 0
            assert deq[i] == 0.0
        err += (int(q[i]) - rec) ** 2
    assert err == info["err_int"]
    assert info["sse_quant_pred"] <= t * (1 + 1e-15) or t < 0


def test_frequency_tables_are_normalised():
    b = synth.random_core((20, 30, 40), seed=3).ravel()
    data, info = Q.compress_core(b, 1e-6 * float(np.dot(b, b)), 256)
    nplanes = int.from_bytes(data[48:52], "little")
    assert nplanes == 64 - info["p_star"]
    f = np.frombuffer(data, "<u2", nplanes * 17, 56).reshape(nplanes, 17)
    for row in f:
        assert row.sum() in (0, 4096)


def test_nothing_encoded_when_target_exceeds_core_energy():
    b = np.array([3.0, -1.0, 0.5])
    data, info = Q.compress_core(b, 100.0, 32)
    assert info["p_star"] == 64
    _, _, deq = Q.decode(data)
    assert np.all(deq == 0)


def test_corrupt_streams_are_rejected():
    b = synth.random_core((10, 10, 10), seed=4).ravel()
    data, _ = Q.compress_core(b, 1e-8 * float(np.dot(b, b)), 64)
    with pytest.raises(ValueError):
        Q.decode(b"XTCQ" + data[4:])
    with pytest.raises(ValueError):
        Q.decode(data[: len(data) // 2])


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3, 1e-4])
def test_full_pipeline_error_within_two_percent(eps):
    x = synth.lowrank_tucker((40, 36, 32), (6, 5, 7), noise="relative", noise_level=1e-3, seed=21)
    stream, info = P.compress(x, eps)
    xh = P.decompress(stream)
    re = np.linalg.norm(x - xh) / np.linalg.norm(x)
    assert 0.98 * eps <= re <= eps * (1 + 1e-12), re
    # Pythagoras of the truncation and quantization errors (complementary patterns)
    sse = float(np.sum((x - xh) ** 2))
    assert abs(sse - (info["sse_trunc"] + info["sse_quant_pred"])) <= 1e-6 * sse
