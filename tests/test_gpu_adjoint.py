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


def _decoded_point(P, n):
    """Core and factors decoded from a compressed stream of the turbulence-like
    field at rel_eps 1e-3: the point where a decompression is differentiated
    (residual ~ rel_eps ||X||)."""
    import synth
    from oracle import pipeline as OP
    x = synth.turbulence(n, device=torch.device("cuda"))
    c = P.atc_compress(x, 1e-3, precision=P.PREC_SPLIT_BF16)
    h = OP.parse(c.stream_bytes())
    ranks, perm = h["ranks"], h["perm"]
    vec = P.atc_dequantize_core(h["core_stream"], int(np.prod(ranks)))
    core = torch.permute(vec.reshape([ranks[p] for p in perm]), tuple(int(i) for i in np.argsort(perm))).contiguous()
    facs = [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in h["factors"]]
    return x, core.float(), [u.float() for u in facs]


def _torch_expand(G, Us, skip=None):
    y = G
    for m in range(len(Us)):
        if m != skip:
            y = torch.movedim(torch.tensordot(Us[m], y, dims=([1], [m])), 0, m)
    return y


def test_decompression_gradient_turbulence(P):
    """L = ||X_hat - X||^2 at the decoded point of a 128^3 turbulence-like field
    (full multilinear rank): FP32 parameters, FP64 products (precision FP64):
    gradients against the FP64 definitions.  X_hat is returned in FP32, so dY =
    2 (X_hat - X) carries a rounding of ~2^-24 ||X|| against a residual of
    ~1e-3 ||X||: relative gradient error ~1e-4 at most."""
    x, core, facs = _decoded_point(P, 128)
    G64, U64 = core.double(), [u.double() for u in facs]
    dY = 2.0 * (_torch_expand(G64, U64) - x.double())
    rG = dY
    for m in range(3):
        rG = torch.movedim(torch.tensordot(U64[m].t(), rG, dims=([1], [m])), 0, m)
    rU = []
    for k in range(3):
        Z = _torch_expand(G64, U64, skip=k)
        rU.append(torch.movedim(dY, k, 0).reshape(dY.shape[k], -1) @ torch.movedim(Z, k, 0).reshape(Z.shape[k], -1).t())
    g = core.clone().requires_grad_(True)
    us = [u.clone().requires_grad_(True) for u in facs]
    loss = torch.sum((P.tucker_expand(g, us, precision=P.PREC_FP64) - x).double() ** 2)
    loss.backward()
    rel = lambda a, b: float(torch.linalg.vector_norm(a.double() - b) / torch.linalg.vector_norm(b))
    assert rel(g.grad, rG) <= 1e-4
    for u, r in zip(us, rU):
        assert rel(u.grad, r) <= 1e-4
    # central difference of the FP64 loss along a random direction against the FP64 gradient
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    vG = torch.randn(G64.shape, generator=gen, device="cuda", dtype=torch.float64)
    vU = [torch.randn(u.shape, generator=gen, device="cuda", dtype=torch.float64) for u in U64]

    def L(h):
        return float(((_torch_expand(G64 + h * vG, [u + h * v for u, v in zip(U64, vU)]) - x.double()) ** 2).sum())
    h = 1e-6 * float(torch.linalg.vector_norm(G64)) / float(torch.linalg.vector_norm(vG))
    fd = (L(h) - L(-h)) / (2 * h)
    an = float((rG * vG).sum()) + sum(float((r * v).sum()) for r, v in zip(rU, vU))
    assert abs(fd - an) <= 1e-2 * abs(fd)
