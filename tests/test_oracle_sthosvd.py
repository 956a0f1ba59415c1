"""Pins of the FP64 ST-HOSVD oracle against facts the paper and linear algebra fix.

Each test checks the oracle against something other than itself: exact
recovery of a tensor built with a known multilinear rank, orthonormality,
norm preservation (Section 3.1), the truncation-error identity of Theorem 6.4
of the cited ST-HOSVD paper (quoted at the end of Section 4.1.3), the d = 2
special case (truncated SVD, Eckart-Young), singular values of independently
formed unfoldings (LAPACK SVD, a different routine from the eigensolver) and
brute force on the rank rule and the decompression order.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

import synth
from oracle import sthosvd as O


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def c0():
    return synth.lowrank_tucker()


def test_exact_multilinear_rank_recovered():
    x = synth.lowrank_tucker(noise=None)
    res = O.sthosvd(x, 1e-2)
    assert res["ranks"] == [8, 8, 8]
    xh = O.reconstruct(res["core"], res["factors"])
    assert np.linalg.norm(x - xh) / np.linalg.norm(x) <= 1e-13


def test_relative_noise_reading_gives_rank_8(c0):
    res = O.sthosvd(c0, 1e-2)
    assert res["ranks"] == [8, 8, 8]


def test_factors_orthonormal(c0):
    res = O.sthosvd(c0, 1e-3)
    for u in res["factors"]:
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-13


def test_core_norm_plus_discarded_equals_input_norm(c0):
    for eps in (1e-1, 1e-2, 1e-3):
        res = O.sthosvd(c0, eps)
        lhs = float(np.sum(res["core"] ** 2)) + res["sse_trunc"]
        assert _rel(lhs, float(np.sum(c0.astype(np.float64) ** 2))) <= 1e-12


@pytest.mark.parametrize("eps,rtmss,rule", [(1e-2, 0.5, "static"), (3e-1, 1.0, "static"),
                                            (2e-1, 1.0, "adaptive"), (1e-3, 0.5, "adaptive")])
def test_truncation_error_equals_discarded_eigenvalues(eps, rtmss, rule):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((12, 10, 14)) + synth.lowrank_tucker((12, 10, 14), (3, 3, 3), noise=None, seed=3)
    res = O.sthosvd(x, eps, rtmss=rtmss, rank_rule=rule)
    xh = O.reconstruct(res["core"], res["factors"])
    lhs = float(np.sum((x - xh) ** 2))
    nx = float(np.sum(x * x))
    assert abs(lhs - res["sse_trunc"]) <= 1e-10 * nx
    if lhs >= 1e-4 * nx:
        assert _rel(res["sse_trunc"], lhs) <= 1e-10
    assert res["sse_trunc"] <= res["budget"] * (1 + 1e-15)


def test_order2_is_truncated_svd():
    rng = np.random.default_rng(11)
    a = rng.standard_normal((40, 25)) @ np.diag(np.geomspace(1, 1e-4, 25)) @ rng.standard_normal((25, 25))
    eps = 1e-2
    res = O.sthosvd(a, eps, rtmss=1.0)
    s = np.linalg.svd(a, compute_uv=False)
    # mode 1 (length 25) is processed first: its eigenvalues are sigma^2
    assert res["order"] == [1, 0]
    lam = res["eigvals"][1]
    np.testing.assert_allclose(lam[: len(s)], s ** 2, rtol=1e-9, atol=1e-12 * s[0] ** 2)
    budget = res["budget"] / 2
    r_expect = next(r for r in range(1, 26) if float(np.sum(s[r:] ** 2)) <= budget)
    assert res["ranks"][1] == r_expect
    xh = O.reconstruct(res["core"], res["factors"])
    # Eckart-Young: the result is the best approximation of rank rho = min(r0, r1)
    # (mode 0 sees the kept sigma^2 and may drop more), error = sum_{j >= rho} sigma_j^2
    rho = min(res["ranks"])
    assert _rel(float(np.sum((a - xh) ** 2)), float(np.sum(s[rho:] ** 2))) <= 1e-8
    assert np.linalg.matrix_rank(xh) == rho


def test_eigenvalues_are_squared_singular_values_of_each_unfolding():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 6, 7))
    res = O.sthosvd(x, 0.3, rtmss=1.0)
    b = x.copy()
    for m in res["order"]:
        mat = np.moveaxis(b, m, 0).reshape(b.shape[m], -1)  # formed independently of the oracle
        s = np.linalg.svd(mat, compute_uv=False)
        lam = res["eigvals"][m]
        np.testing.assert_allclose(lam[: len(s)], s ** 2, rtol=1e-10, atol=1e-12 * s[0] ** 2)
        u = res["factors"][m]
        b = np.moveaxis(np.einsum("ir,i...->r...", u, np.moveaxis(b, m, 0)), 0, m)


def test_rank_rule_brute_force():
    rng = np.random.default_rng(9)
    for _ in range(300):
        n = int(rng.integers(1, 9))
        lam = np.sort(rng.integers(0, 20, size=n).astype(np.float64))[::-1]
        budget = float(rng.integers(0, 40))
        r = O.choose_rank(lam, budget)
        fr = [Fraction(v) for v in lam]
        ok = [rr for rr in range(1, n + 1) if sum(fr[rr:], Fraction(0)) <= Fraction(budget)]
        assert r == min(ok)


def test_processing_order_increasing_length_ties_by_index():
    assert O.processing_order([256, 256, 256]) == [0, 1, 2]
    assert O.processing_order([512, 512, 224]) == [2, 0, 1]
    assert O.processing_order([7, 3, 7, 3]) == [1, 3, 0, 2]
    assert O.processing_order([5, 4], mode_order=[0, 1]) == [0, 1]
    with pytest.raises(ValueError):
        O.processing_order([5, 4], mode_order=[0, 0])


def test_decompression_order_brute_force():
    dims, ranks = [64, 30, 100], [8, 20, 5]
    costs = {}
    for p in itertools.permutations(range(3)):
        c = 0
        for i in range(3):
            c += int(np.prod([dims[p[j]] for j in range(i + 1)])) * int(np.prod([ranks[p[j]] for j in range(i, 3)]))
        costs[p] = c
    best = min(costs.values())
    assert costs[tuple(O.decompression_order(dims, ranks))] == best


def test_mode_order_does_not_change_the_error_guarantee(c0):
    for order in ([2, 1, 0], [1, 0, 2]):
        res = O.sthosvd(c0, 1e-2, mode_order=order)
        xh = O.reconstruct(res["core"], res["factors"])
        assert float(np.sum((c0 - xh) ** 2)) <= res["budget"] * (1 + 1e-9)


def test_rtmss_zero_keeps_full_rank():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((6, 5, 4))
    res = O.sthosvd(x, 1e-1, rtmss=0.0)
    assert res["ranks"] == [6, 5, 4]


def test_invalid_arguments():
    x = np.ones((2, 2))
    for eps in (0.0, -1.0, 1.5):
        with pytest.raises(ValueError):
            O.sthosvd(x, eps)
    with pytest.raises(ValueError):
        O.sthosvd(x, 0.1, rtmss=1.5)


def test_storage_order_hand_worked_cases():
    """Supplement S.2: the core's modes are stored in order of increasing size
    (the shortest mode first, i.e. slowest-varying in the lexicographic
    vectorisation), ties by lower index.  Worked by hand."""
    assert O.storage_order([19, 18, 21]) == [1, 0, 2]
    assert O.storage_order([8, 8, 8]) == [0, 1, 2]          # all equal: identity
    assert O.storage_order([5, 3, 5]) == [1, 0, 2]          # tie between 0 and 2 keeps 0 first
    assert O.storage_order([4, 4, 2]) == [2, 0, 1]
    assert O.storage_order([7, 2, 7, 1]) == [3, 1, 0, 2]    # 4-D with a tie
    assert O.storage_order([3, 3, 3, 3]) == [0, 1, 2, 3]
    assert O.storage_order([9, 1]) == [1, 0]
    assert O.storage_order([6]) == [0]
    # decreasing sizes reverse completely
    assert O.storage_order([40, 30, 20, 10]) == [3, 2, 1, 0]


def test_storage_order_brute_force():
    """Against brute force over all d! permutations: the storage order is the
    lexicographically first permutation whose permuted sizes do not decrease
    (a permutation search, not a sort)."""
    rng = np.random.default_rng(23)
    for _ in range(200):
        d = int(rng.integers(1, 6))
        ranks = [int(v) for v in rng.integers(1, 5, size=d)]
        ok = [p for p in itertools.permutations(range(d))
              if all(ranks[p[i]] <= ranks[p[i + 1]] for i in range(d - 1))]
        assert O.storage_order(ranks) == list(min(ok))


def test_vectorisation_in_storage_order_by_hand():
    """The vectorised core in storage order, written out with explicit loops:
    ranks (4, 2, 3) give storage order (1, 2, 0), i.e. the core is read as
    b[a, b, c] at position b*12 + c*4 + a (Section 3.3 vectorisation,
    lexicographic, last storage index fastest)."""
    from oracle import pipeline as OP
    core = np.arange(24, dtype=np.float64).reshape(4, 2, 3) * 1.5 - 7.0
    perm = O.storage_order(list(core.shape))
    assert perm == [1, 2, 0]
    vec = OP.vectorize_core(core, perm)
    for a in range(4):
        for b in range(2):
            for c in range(3):
                assert vec[b * 12 + c * 4 + a] == core[a, b, c]
    # and back
    assert np.array_equal(OP.devectorize_core(vec, list(core.shape), perm), core)
