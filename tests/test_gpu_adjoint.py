"""Differentiable Tucker expansion X_hat = G x_1 U_1 ... x_d U_d (the
reconstruction of Section 4.1.1 / 4.3) and its hand-written adjoint, through
the C ABI: against the FP64 definitions written out with einsum, against
finite differences (torch.autograd.gradcheck), and the split-precision
(tensor-core) variant against FP64.

Definitions (d = 3, indices i, j, k of X_hat and a, b, c of G):
  X_hat[i,j,k] = sum_{abc} G[a,b,c] U1[i,a] U2[j,b] U3[k,c]
  dL/dG[a,b,c] = sum_{ijk} dY[i,j,k] U1[i,a] U2[j,b] U3[k,c]
  dL/dU1[i,a]  = sum_{jkbc} dY[i,j,k] G[a,b,c] U2[j,b] U3[k,c]      (and likewise for U2, U3)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2107_01384_gb300 as P
    return P


def ref_forward(G, Us):
    return np.einsum("abc,ia,jb,kc->ijk", G, *Us)


def ref_grads(dY, G, Us):
    U1, U2, U3 = Us
    dG = np.einsum("ijk,ia,jb,kc->abc", dY, U1, U2, U3)
    d1 = np.einsum("ijk,abc,jb,kc->ia", dY, G, U2, U3)
    d2 = np.einsum("ijk,abc,ia,kc->jb", dY, G, U1, U3)
    d3 = np.einsum("ijk,abc,ia,jb->kc", dY, G, U1, U2)
    return dG, [d1, d2, d3]


def problem(dims, ranks, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(ranks)
    Us = [rng.standard_normal((n, r)) / np.sqrt(n) for n, r in zip(dims, ranks)]
    dY = rng.standard_normal(dims)
    return G, Us, dY


CASES = [((9, 7, 11), (4, 3, 5), 0), ((64, 40, 33), (8, 6, 7), 1), ((130, 70, 20), (31, 9, 20), 2)]


@pytest.mark.parametrize("dims,ranks,seed", CASES)
def test_forward_and_adjoint_fp64(P, dims, ranks, seed):
    G, Us, dY = problem(dims, ranks, seed)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    xh = P.atc_tucker_expand(cu(G), [cu(u) for u in Us]).cpu().numpy()
    ref = ref_forward(G, Us)
    assert np.abs(xh - ref).max() <= 1e-12 * np.abs(ref).max()
    dG, dU = P.atc_tucker_expand_adjoint(cu(dY), cu(G), [cu(u) for u in Us])
    rG, rU = ref_grads(dY, G, Us)
    assert np.abs(dG.cpu().numpy() - rG).max() <= 1e-11 * np.abs(rG).max()
    for a, b in zip(dU, rU):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-11 * np.abs(b).max()


def test_gradcheck_finite_differences(P):
    """Central finite differences of the FP64 forward against the adjoint."""
    G, Us, _ = problem((6, 5, 4), (3, 2, 3), 3)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda().requires_grad_(True)
    inputs = (cu(G), cu(Us[0]), cu(Us[1]), cu(Us[2]))
    f = lambda g, u1, u2, u3: P.tucker_expand(g, [u1, u2, u3])
    assert torch.autograd.gradcheck(f, inputs, eps=1e-6, atol=1e-8, rtol=1e-6)


def test_loss_gradient_matches_definition(P):
    """L = ||X_hat - X||^2: autograd through the Function equals 2 (X_hat - X)
    pushed through the definitions."""
    G, Us, _ = problem((40, 36, 30), (6, 5, 7), 4)
    X = np.random.default_rng(5).standard_normal((40, 36, 30))
    g = torch.from_numpy(G).cuda().requires_grad_(True)
    us = [torch.from_numpy(u).cuda().requires_grad_(True) for u in Us]
    xh = P.tucker_expand(g, us)
    loss = ((xh - torch.from_numpy(X).cuda()) ** 2).sum()
    loss.backward()
    dY = 2.0 * (ref_forward(G, Us) - X)
    rG, rU = ref_grads(dY, G, Us)
    assert np.abs(g.grad.cpu().numpy() - rG).max() <= 1e-10 * np.abs(rG).max()
    for u, r in zip(us, rU):
        assert np.abs(u.grad.cpu().numpy() - r).max() <= 1e-10 * np.abs(r).max()


@pytest.mark.parametrize("prec", [1, 2])
def test_split_precision_adjoint(P, prec):
    """Tensor-core variant (FP32 data, exact slice products, one rounding per
    output): within FP32 level of the FP64 definitions."""
    G, Us, dY = problem((64, 40, 33), (8, 6, 7), 6)
    G32 = torch.from_numpy(G.astype(np.float32)).cuda()
    us = [torch.from_numpy(u).cuda() for u in Us]
    dy32 = torch.from_numpy(dY.astype(np.float32)).cuda()
    xh = P.atc_tucker_expand(G32, us, precision=prec).cpu().numpy().astype(np.float64)
    ref = ref_forward(G.astype(np.float32).astype(np.float64), Us)
    assert np.abs(xh - ref).max() <= 1e-5 * np.abs(ref).max()
    dG, dU = P.atc_tucker_expand_adjoint(dy32, G32, us, precision=prec)
    rG, rU = ref_grads(dY.astype(np.float32).astype(np.float64), G.astype(np.float32).astype(np.float64), Us)
    assert np.abs(dG.cpu().numpy() - rG).max() <= 1e-5 * np.abs(rG).max()
    for a, b in zip(dU, rU):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-5 * np.abs(b).max()
