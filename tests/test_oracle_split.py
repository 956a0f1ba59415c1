"""Pins of the oracle's split bit-plane truncation (supplement S.3) against
literal bit-by-bit simulations in Python integers.

The last plane p* (from the walk in coefficient order, Section 3.3) is split
into its leading bits (coefficients not yet significant above p*) and its
trailing bits (significant ones).  The category whose bits were more efficient
on plane p* + 1 -- SSE reduction per encoded bit, the leading bits costing their
rANS bytes plus one sign bit per leading 1, the trailing bits one raw bit each
-- is walked first, in coefficient order, then the other; the first bit at
which the tracked error meets the target gives (i_lead, i_trail).
"""
import struct
from fractions import Fraction

import numpy as np
import pytest

from oracle import quant as Q


def _target_int(t, k):
    if t < 0:
        return None
    return int(Fraction(t) * Fraction(2) ** (2 * k) // 1)


class _Sim:
    """Decoder-side state of a literal bit-plane walk: bits known so far and
    each coefficient's lowest decoded plane (Section 4.3 reconstruction)."""

    def __init__(self, q):
        self.q = [int(v) for v in q]
        self.known = [0] * len(q)
        self.lowest = [64] * len(q)

    def err(self, i):
        if self.known[i] == 0:
            return self.q[i] ** 2
        p = self.lowest[i]
        rec = self.known[i] + ((1 << (p - 1)) if p >= 1 else 0)
        return (self.q[i] - rec) ** 2

    def total(self):
        return sum(self.err(i) for i in range(len(self.q)))

    def reveal(self, i, p):
        self.known[i] |= self.q[i] & (1 << p)
        self.lowest[i] = p

    def significant_above(self, i, p):
        return p < 63 and (self.q[i] >> (p + 1)) != 0


def _literal_standard(q, tint):
    sim = _Sim(q)
    n = len(q)
    if tint is not None and sim.total() <= tint:
        return 64, n - 1, sim.total()
    for p in range(63, -1, -1):
        for i in range(n):
            sim.reveal(i, p)
            if tint is not None and sim.total() <= tint:
                return p, i, sim.total()
    return 0, n - 1, sim.total()


def _sim_through(q, p_last):
    """State after every bit of planes 63 .. p_last."""
    sim = _Sim(q)
    for p in range(63, p_last - 1, -1):
        for i in range(len(q)):
            sim.reveal(i, p)
    return sim


def _literal_efficiencies(q, p):
    """Exact SSE reductions of plane p's leading and trailing bits (encoded
    whole after planes 63 .. p + 1) and the counts of leading ones and of
    trailing bits."""
    sim = _sim_through(q, p + 1) if p < 63 else _Sim(q)
    before = [sim.err(i) for i in range(len(q))]
    cat = [sim.significant_above(i, p) for i in range(len(q))]
    for i in range(len(q)):
        sim.reveal(i, p)
    after = [sim.err(i) for i in range(len(q))]
    d_lead = sum(b - a for b, a, c in zip(before, after, cat) if not c)
    d_trail = sum(b - a for b, a, c in zip(before, after, cat) if c)
    ones = sum(1 for i, c in enumerate(cat) if not c and (sim.q[i] >> p) & 1)
    trail = sum(1 for c in cat if c)
    return d_lead, d_trail, ones, trail


def _plane_rans_bytes_from_stream(q, s, k, p, block_size):
    """rANS bytes of plane p encoded whole, read from the size table of a
    stream whose last plane is p (every bit of planes 63 .. p encoded)."""
    n = len(q)
    data = Q.encode(q, s, k, p, n - 1, n - 1, block_size)
    nplanes = 64 - p
    tab = 56 + nplanes * 17 * 2
    nblocks = (n + block_size - 1) // block_size
    total = 0
    for b in range(nblocks):
        rl, _ = struct.unpack_from("<II", data, tab + (b * nplanes + nplanes - 1) * 8)
        total += rl
    return total


def _literal_split(q, s, k, tint, block_size):
    n = len(q)
    p_star, i_star, err = _literal_standard(q, tint)
    if p_star >= 64:
        return p_star, 0, n - 1, n - 1, err
    prio = 0
    if p_star < 63:
        dl, dt, ones, trail = _literal_efficiencies(q, p_star + 1)
        cost_lead = 8 * _plane_rans_bytes_from_stream(q, s, k, p_star + 1, block_size) + ones
        cost_trail = trail
        prio = 0 if dl * cost_trail >= dt * cost_lead else 1
    sim = _sim_through(q, p_star + 1) if p_star < 63 else _Sim(q)
    cat = [sim.significant_above(i, p_star) for i in range(n)]
    order = [0, 1] if prio == 0 else [1, 0]
    for pass_, c in enumerate(order):
        for i in range(n):
            if int(cat[i]) != c:
                continue
            sim.reveal(i, p_star)
            if tint is not None and sim.total() <= tint:
                first = order[0]
                if pass_ == 0:
                    j_first, j_second = i, -1
                else:
                    j_first, j_second = n - 1, i
                il, it = (j_first, j_second) if first == 0 else (j_second, j_first)
                return p_star, prio, il, it, sim.total()
    return p_star, prio, i_star, i_star, err


def _cases(seed, trials):
    rng = np.random.default_rng(seed)
    for trial in range(trials):
        n = int(rng.integers(1, 14))
        b = rng.standard_normal(n) * np.exp(-rng.uniform(0, 10, n))
        if trial % 5 == 0:
            b[rng.integers(0, n, size=max(1, n // 3))] = 0.0
        yield trial, b


def test_split_breakpoint_matches_literal_walk():
    seen_prio = set()
    seen_second = 0
    for trial, b in _cases(11, 80):
        k = Q.scale_exponent(b)
        q, s = Q.quantize(b, k)
        nb = float(np.dot(b, b))
        for frac in (1.0, 0.3, 3e-2, 1e-3, 1e-6, 1e-11, 0.0, -1.0):
            t = frac * nb
            got = Q.split_breakpoint(q, s, t, k, 32)
            want = _literal_split(q, s, k, _target_int(t, k), 32)
            assert got == want, (trial, frac, got, want)
            seen_prio.add(got[1])
            if got[0] < 64 and got[2] != got[3] and -1 not in (got[2], got[3]):
                seen_second += 1
    # both priorities and second-pass breakpoints occur in this sample
    assert seen_prio == {0, 1}
    assert seen_second > 0


def test_plane_efficiencies_match_literal_reductions():
    for trial, b in _cases(5, 40):
        k = Q.scale_exponent(b)
        q, s = Q.quantize(b, k)
        for p in (63, 62, 60, 55, 40, 1, 0):
            e = Q.plane_efficiencies(q, s, p, 32)
            dl, dt, ones, trail = _literal_efficiencies(q, p)
            assert (e["d_lead"], e["d_trail"]) == (dl, dt), (trial, p)
            assert e["cost_trail"] == trail
            assert e["cost_lead"] == 8 * _plane_rans_bytes_from_stream(q, s, k, p, 32) + ones


@pytest.mark.parametrize("n,bs,frac,seed", [(700, 32, 1e-3, 0), (5000, 64, 1e-5, 1), (20000, 4096, 1e-7, 2)])
def test_split_never_worse_than_single_breakpoint(n, bs, frac, seed):
    """Both truncations stop at the first bit meeting the same target on the
    same plane; the split one meets it as well (its tracked error is <= the
    target whenever the single breakpoint's is)."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(n) * np.exp(-np.arange(n) / (n / 6))
    t = frac * float(np.dot(b, b))
    d1, i1 = Q.compress_core(b, t, bs, split=True)
    d0, i0 = Q.compress_core(b, t, bs, split=False)
    assert i1["p_star"] == i0["p_star"]
    assert i1["err_int"] <= _target_int(t, i1["k"])
    assert i0["err_int"] <= _target_int(t, i0["k"])
    for data in (d0, d1):
        _, _, deq = Q.decode(data)
        assert float(np.sum((deq - b) ** 2)) <= t * (1 + 1e-9)
