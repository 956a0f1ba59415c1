"""Plain FP64 CPU oracle for the ST-HOSVD mode loop (TEST INFRASTRUCTURE ONLY).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path (the CUDA library and its
Python binding) never calls it.

Everything here follows the paper's definitions step by step, in float64, with
NumPy's matmul / tensordot / eigh as library primitives:

* Section 3.1  -- mode-k matricization X_(k) and the mode-k product
                  Y = U ._k X  <=>  Y_(k) = U X_(k).
* Algorithm 1  -- ST-HOSVD: per mode, factor from the singular vectors of the
                  current unfolding, rank choice, projection.  The left singular
                  vectors / values are taken from the eigendecomposition of the
                  Gram matrix B_(k) B_(k)^T (lambda = sigma^2).
* Section 4.1.1 -- modes processed in order of increasing length (ties: lower
                  index first), or a user-given order.
* Section 4.1.3 -- TargetSSE_total = rel_eps^2 ||X||^2,
                  TargetSSE_ST-HOSVD = RTMSS * TargetSSE_total (default 0.5);
                  actual truncation SSE = sum of the discarded squared singular
                  values over all modes (Theorem 6.4 of the cited ST-HOSVD paper).
* Rank rule    -- the paper defers to Section 6.3 of the cited ST-HOSVD paper.
                  Reading used here ("static"): every one of the d modes gets the
                  budget TargetSSE_ST-HOSVD / d and keeps the smallest r >= 1 whose
                  discarded eigenvalue sum fits.  Option "adaptive" hands the unused
                  budget on: budget_i = (TargetSSE_ST-HOSVD - used) / (modes left).
* Section 4.1.1 -- decompression order minimising sum_i n_p1..n_pi r_pi..r_pd,
                  by exhaustive search.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "norm2",
    "processing_order",
    "unfold",
    "mode_gram",
    "eig_descending",
    "tail_sums",
    "choose_rank",
    "ttm_project",
    "ttm_expand",
    "sthosvd",
    "reconstruct",
    "decompression_order",
    "storage_order",
]


def norm2(x) -> float:
    """||X||^2 = <X, X> in float64 (Section 3.1, Euclidean inner product)."""
    v = np.asarray(x, dtype=np.float64).ravel()
    return float(np.dot(v, v))


def processing_order(dims, mode_order=None):
    """Mode processing order (Section 4.1.1): increasing mode length, ties by index."""
    d = len(dims)
    if mode_order is not None:
        order = [int(m) for m in mode_order]
        if sorted(order) != list(range(d)):
            raise ValueError("mode_order must be a permutation of range(d)")
        return order
    return sorted(range(d), key=lambda i: (dims[i], i))


def unfold(b: np.ndarray, k: int) -> np.ndarray:
    """Mode-k matricization B_(k): row i_k, columns = the remaining indices in
    lexicographic order (Section 3.1)."""
    return np.moveaxis(b, k, 0).reshape(b.shape[k], -1)


def mode_gram(b: np.ndarray, k: int) -> np.ndarray:
    """G = B_(k) B_(k)^T in float64."""
    m = unfold(np.asarray(b, dtype=np.float64), k)
    return m @ m.T


def eig_descending(g: np.ndarray):
    """Eigen-pairs of the symmetric Gram matrix, eigenvalues descending and
    clamped at zero (a Gram matrix is positive semi-definite; negative values
    are rounding).  Sign convention: the entry of largest magnitude in each
    eigenvector (first one on ties) is made positive."""
    lam, v = np.linalg.eigh(np.asarray(g, dtype=np.float64))
    order = np.argsort(-lam, kind="stable")
    lam = np.maximum(lam[order], 0.0)
    v = v[:, order].copy()
    for j in range(v.shape[1]):
        i = int(np.argmax(np.abs(v[:, j])))
        if v[i, j] < 0:
            v[:, j] = -v[:, j]
    return lam, v


def tail_sums(lam) -> np.ndarray:
    """t[r] = sum_{j >= r} lam[j] (0-based), summed from the smallest value
    upward, t[n] = 0.  t[r] is the energy discarded when keeping r columns."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    t = np.zeros(n + 1, dtype=np.float64)
    acc = 0.0
    for j in range(n - 1, -1, -1):
        acc += float(lam[j])
        t[j] = acc
    return t


def choose_rank(lam, budget: float) -> int:
    """Smallest r >= 1 with discarded energy t[r] <= budget."""
    t = tail_sums(lam)
    n = len(lam)
    for r in range(1, n + 1):
        if t[r] <= budget:
            return r
    return n


def ttm_project(b: np.ndarray, u: np.ndarray, k: int) -> np.ndarray:
    """Y = U^T ._k B, i.e. Y_(k) = U^T B_(k) (Algorithm 1, projection step)."""
    y = np.tensordot(np.asarray(u, dtype=np.float64).T, b, axes=([1], [k]))
    return np.moveaxis(y, 0, k)


def ttm_expand(b: np.ndarray, u: np.ndarray, k: int) -> np.ndarray:
    """Y = U ._k B, i.e. Y_(k) = U B_(k) (decompression)."""
    y = np.tensordot(np.asarray(u, dtype=np.float64), b, axes=([1], [k]))
    return np.moveaxis(y, 0, k)


def sthosvd(x, rel_eps: float, rtmss: float = 0.5, mode_order=None, rank_rule: str = "static"):
    """ST-HOSVD with error-driven rank choice (Algorithm 1, Section 4.1.3).

    Returns a dict with the core (float64, modes in their original positions),
    the factors U_k (n_k x r_k), the ranks, the processing order, ||X||^2,
    TargetSSE_total, the ST-HOSVD budget, the actual truncation SSE and the
    per-mode eigenvalues and discarded energies."""
    x = np.asarray(x, dtype=np.float64)
    if not (0.0 < rel_eps <= 1.0):
        raise ValueError("rel_eps must lie in (0, 1]")
    if not (0.0 <= rtmss <= 1.0):
        raise ValueError("rtmss must lie in [0, 1]")
    d = x.ndim
    dims = list(x.shape)
    nrm2 = norm2(x)
    target_total = rel_eps * rel_eps * nrm2
    budget_total = rtmss * target_total
    order = processing_order(dims, mode_order)
    b = x
    factors = [None] * d
    ranks = [None] * d
    eigvals = [None] * d
    discarded = [0.0] * d
    used = 0.0
    for step, m in enumerate(order):
        g = mode_gram(b, m)
        lam, v = eig_descending(g)
        if rank_rule == "static":
            budget = budget_total / d
        elif rank_rule == "adaptive":
            budget = (budget_total - used) / (d - step)
        else:
            raise ValueError(f"unknown rank rule {rank_rule!r}")
        r = choose_rank(lam, budget)
        t = tail_sums(lam)
        factors[m] = np.ascontiguousarray(v[:, :r])
        ranks[m] = r
        eigvals[m] = lam
        discarded[m] = float(t[r])
        used += float(t[r])
        b = ttm_project(b, factors[m], m)
    return {
        "core": np.ascontiguousarray(b),
        "factors": factors,
        "ranks": ranks,
        "order": order,
        "norm2": nrm2,
        "target_sse": target_total,
        "budget": budget_total,
        "sse_trunc": used,
        "discarded": discarded,
        "eigvals": eigvals,
    }


def decompression_order(dims, ranks):
    """Order p minimising sum_i n_p1..n_pi * r_pi..r_pd (Section 4.1.1), by
    exhaustive search over all d! orders; the first minimal order in
    lexicographic permutation order wins ties."""
    d = len(dims)
    best, best_cost = None, None
    for p in itertools.permutations(range(d)):
        cost = 0
        for i in range(d):
            c = 1
            for j in range(i + 1):
                c *= int(dims[p[j]])
            for j in range(i, d):
                c *= int(ranks[p[j]])
            cost += c
        if best_cost is None or cost < best_cost:
            best, best_cost = list(p), cost
    return best


def reconstruct(core, factors, order=None):
    """X_hat = core x_1 U_1 ... x_d U_d (order only changes the cost)."""
    b = np.asarray(core, dtype=np.float64)
    d = b.ndim
    if order is None:
        order = decompression_order([u.shape[0] for u in factors], [u.shape[1] for u in factors])
    for m in order:
        b = ttm_expand(b, factors[m], m)
    return b


def storage_order(ranks):
    """Mode storage order of the core before vectorisation (supplement, Section
    S.2): increasing mode size, ties by index."""
    return sorted(range(len(ranks)), key=lambda i: (ranks[i], i))
