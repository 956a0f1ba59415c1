"""GPU parity of the split-precision tensor-core kernels (tcgen05) against the
FP64 oracle, through the C ABI.

Error model (written out so the tolerances are derivable):
* x = h + l + rho with h, l 16-bit halves.  bf16: |rho| <= 2^-17 |x| and the
  dropped l*l' term <= 2^-16 |x y|; fp16 (pre-scaled, 11-bit halves): 2^-23 and
  2^-22.  So one split product is within c * 2^-15 |x y| (bf16) or
  c * 2^-21 |x y| (fp16) of x*y, c <= 2.
* Accumulation in FP32 inside one CTA adds about 2^-24 * sqrt(K_chunk) of
  the sum of |products|; partial sums are combined in FP64.
Hence for the Gram matrix |G - G_ref|_ij <= tol * sqrt(G_ii G_jj) with
tol = 2^-13 (bf16) or 2^-18 (fp16), and for the projection
|Y - Y_ref| <= tol * ||x_gamma|| per output column.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import sthosvd as O  # noqa: E402

TOL = {1: 2.0 ** -13, 2: 2.0 ** -18}


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2107_01384_gb300 as P
    return P


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


GRAM_CASES = [((64, 64, 64), 0, np.float64), ((64, 64, 64), 1, np.float64), ((64, 64, 64), 2, np.float64),
              ((256, 256, 16), 0, np.float32), ((16, 256, 256), 1, np.float32), ((100, 100, 256), 2, np.float32),
              ((37, 129, 5), 1, np.float32), ((200, 7), 0, np.float32), ((1, 200, 1000), 1, np.float32),
              ((5, 17, 3), 1, np.float32), ((3, 256, 40), 1, np.float32), ((70, 224), 1, np.float32)]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dims,mode,dtype", GRAM_CASES)
def test_gram_split(P, dims, mode, dtype, prec):
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(dims) * np.exp(rng.uniform(-2, 2, size=dims))).astype(dtype)
    L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
    g = P.atc_gram(cuda(x), L, n, R, prec).cpu().numpy()
    ref = O.mode_gram(x, mode)
    d = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    err = np.abs(g - ref) / np.maximum(d, 1e-300)
    assert err.max() <= TOL[prec], err.max()
    assert np.array_equal(g, g.T)


TTM_CASES = [((64, 64, 64), 0, 8, np.float64), ((64, 64, 64), 1, 8, np.float64), ((64, 64, 64), 2, 13, np.float32),
             ((256, 256, 16), 0, 30, np.float32), ((16, 256, 256), 1, 20, np.float32),
             ((100, 100, 256), 2, 200, np.float32), ((37, 129, 5), 1, 20, np.float32), ((300, 7), 1, 7, np.float32),
             ((3, 100, 1), 1, 1, np.float32), ((9, 70, 33), 1, 64, np.float32), ((50, 256), 1, 256, np.float32)]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dims,mode,r,dtype", TTM_CASES)
def test_ttm_split(P, dims, mode, r, dtype, prec):
    rng = np.random.default_rng(8)
    x = rng.standard_normal(dims).astype(dtype)
    u, _ = np.linalg.qr(rng.standard_normal((dims[mode], r)))
    L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
    y = P.atc_ttm(cuda(x), L, n, R, cuda(u), r, expand=False, precision=prec, out_dtype=torch.float32).cpu().numpy()
    ref = O.ttm_project(x.astype(np.float64), u, mode)
    colnorm = np.sqrt(np.sum(np.moveaxis(x.astype(np.float64), mode, 0) ** 2, axis=0))  # ||x_gamma||
    err = np.abs(np.moveaxis(y.reshape(ref.shape), mode, 0) - np.moveaxis(ref, mode, 0)) / np.maximum(colnorm, 1e-300)
    assert err.max() <= TOL[prec], err.max()


@pytest.mark.parametrize("prec", [1, 2])
def test_ttm_split_expand(P, prec):
    rng = np.random.default_rng(9)
    dims = (20, 12, 30)
    u, _ = np.linalg.qr(rng.standard_normal((90, 12)))
    x = rng.standard_normal(dims).astype(np.float32)
    y = P.atc_ttm(cuda(x), 20, 90, 30, cuda(u), 12, expand=True, precision=prec, out_dtype=torch.float32).cpu().numpy()
    ref = O.ttm_expand(x.astype(np.float64), u, 1)
    scale = np.sqrt(np.sum(x.astype(np.float64) ** 2, axis=1))  # per (l, c) column norm of the input
    err = np.abs(y.reshape(ref.shape) - ref) / np.maximum(scale[:, None, :], 1e-300)
    assert err.max() <= TOL[prec], err.max()


def test_split_rejects_unsupported(P):
    x = torch.zeros(2, 1100, 2, device="cuda")
    with pytest.raises(P.AtcError):
        P.atc_gram(x, 2, 1100, 2, 1)


@pytest.mark.parametrize("prec", [1, 2])
def test_pipeline_split_lowrank64(P, prec):
    x = synth.lowrank_tucker()
    ref = O.sthosvd(x, 1e-2)
    c = P.atc_compress(cuda(x), 1e-2, precision=prec)
    assert c.ranks() == ref["ranks"]
    xh = P.atc_decompress(c.stream_bytes()).cpu().numpy()
    re = np.linalg.norm(x - xh) / np.linalg.norm(x)
    assert 0.98e-2 <= re <= 1e-2, re


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_pipeline_split_bumps256(P, prec, eps):
    x = synth.gaussian_bumps()
    ref = O.sthosvd(x, eps)
    c = P.atc_compress(cuda(x), eps, precision=prec)
    assert c.ranks() == ref["ranks"], (c.ranks(), ref["ranks"])
    xh = P.atc_decompress(c.stream_bytes()).cpu().numpy()
    re = np.linalg.norm(x - xh) / np.linalg.norm(x)
    assert 0.98 * eps <= re <= eps, re
