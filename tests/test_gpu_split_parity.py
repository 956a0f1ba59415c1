"""GPU parity of the split-precision tensor-core kernels (tcgen05) against the
FP64 oracle, through the C ABI.

Error model (written out so the tolerances are derivable):
* Each element is read as v = x 2^shift (one power-of-two scale per tensor,
  |v| < 256, 2^-shift * 256 = 2^E <= 2 max|x|) and cut into three integer
  slices, v ~ a0 + a1 2^-8 + a2 2^-16, rounded to nearest: |x - x~| <= 2^(E-25)
  <= 2^-24 M with M = max|x|.  Factors (|U| <= 1) are sliced on the scale 2^8:
  |u - u~| <= 2^-25.
* The tensor cores form all nine slice products, grouped by order into five
  accumulators that stay integers below 2^24, so nothing rounds there; the
  orders are combined in double-float / FP64.
Hence |G - G_ref|_ij <= 2^-24 M sqrt(K) (||x_i|| + ||x_j||) + K 2^-48 M^2, and
for the projection |y - y_ref| <= 2^-24 (M sqrt(n) + sqrt(n) ||x_gamma|| + |y|);
the tests use these bounds with a factor 4.  Exactness tests use data whose
slices are exact: there the results must equal the exact values.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import pipeline as OP  # noqa: E402
from oracle import quant as OQ  # noqa: E402
from oracle import sthosvd as O  # noqa: E402

def ttm_bound(M, K, colnorm, y):
    """|y - y_ref| bound of the error model, for contraction length K."""
    return 4 * 2.0 ** -24 * (M * np.sqrt(K) + np.sqrt(K) * colnorm + np.abs(y))

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
              ((5, 17, 3), 1, np.float32), ((3, 256, 40), 1, np.float32), ((70, 224), 1, np.float32),
              # raw tiles by TMA, sliced in the kernel: ragged n, a K tail, many tile pairs, R = 224
              ((3, 100, 96), 1, np.float32), ((130, 36), 1, np.float32), ((2, 1024, 32), 1, np.float32),
              ((7, 64, 224), 1, np.float32)]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dims,mode,dtype", GRAM_CASES)
def test_gram_split(P, dims, mode, dtype, prec):
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(dims) * np.exp(rng.uniform(-2, 2, size=dims))).astype(dtype)
    L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
    g = P.atc_gram(cuda(x), L, n, R, prec).cpu().numpy()
    ref = O.mode_gram(x, mode)
    M = float(np.abs(x).max()); K = L * R
    rn = np.sqrt(np.diag(ref))
    bound = 2.0 ** -24 * M * np.sqrt(K) * (rn[:, None] + rn[None, :]) + K * 2.0 ** -48 * M * M
    assert np.all(np.abs(g - ref) <= 4 * bound), (np.abs(g - ref) / bound).max()
    assert np.array_equal(g, g.T)


TTM_CASES = [((64, 64, 64), 0, 8, np.float64), ((64, 64, 64), 1, 8, np.float64), ((64, 64, 64), 2, 13, np.float32),
             ((256, 256, 16), 0, 30, np.float32), ((16, 256, 256), 1, 20, np.float32),
             ((100, 100, 256), 2, 200, np.float32), ((37, 129, 5), 1, 20, np.float32), ((300, 7), 1, 7, np.float32),
             ((3, 100, 1), 1, 1, np.float32), ((9, 70, 33), 1, 64, np.float32), ((50, 256), 1, 256, np.float32),
             # raw tiles by TMA: R a power of two below 128, R = 4, R a multiple of 128 with a K tail
             ((10, 96, 64), 1, 24, np.float32), ((40, 50, 4), 1, 9, np.float32), ((2, 130, 384), 1, 17, np.float32),
             ((5, 70, 128), 1, 31, np.float32)]


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
    yr = np.moveaxis(ref, mode, 0)
    err = np.abs(np.moveaxis(y.reshape(ref.shape), mode, 0) - yr)
    bound = ttm_bound(float(np.abs(x).max()), dims[mode], colnorm[None], yr)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("prec", [1, 2])
def test_ttm_split_expand(P, prec):
    rng = np.random.default_rng(9)
    dims = (20, 12, 30)
    u, _ = np.linalg.qr(rng.standard_normal((90, 12)))
    x = rng.standard_normal(dims).astype(np.float32)
    y = P.atc_ttm(cuda(x), 20, 90, 30, cuda(u), 12, expand=True, precision=prec, out_dtype=torch.float32).cpu().numpy()
    ref = O.ttm_expand(x.astype(np.float64), u, 1)
    scale = np.sqrt(np.sum(x.astype(np.float64) ** 2, axis=1))  # per (l, c) column norm of the input
    err = np.abs(y.reshape(ref.shape) - ref)
    bound = ttm_bound(float(np.abs(x).max()), 12, scale[:, None, :], ref)
    assert np.all(err <= bound), (err / bound).max()


EXACT_CASES = [((64, 64, 64), 0), ((64, 64, 64), 2), ((3, 256, 700), 1), ((37, 129, 5), 1), ((1, 200, 1000), 1),
               ((700, 224), 1), ((5, 300, 33), 1), ((3, 100, 96), 1), ((130, 36), 1)]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dims,mode", EXACT_CASES)
def test_gram_split_exact_integer(P, dims, mode, prec):
    """Values on an 8-bit grid: one slice each, so every product and every
    partial sum is an integer below 2^24 and the tensor-core Gram must equal
    the exact FP64 Gram bit for bit (no truncation anywhere)."""
    rng = np.random.default_rng(11)
    x = (rng.integers(-255, 256, size=dims) * 0.125).astype(np.float32)
    x.flat[0] = 255 * 0.125  # max|x| = 31.875 -> shift 3, v = 8 x integer
    L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
    g = P.atc_gram(cuda(x), L, n, R, prec).cpu().numpy()
    ref = O.mode_gram(x.astype(np.float64), mode)
    assert np.array_equal(g, ref), np.abs(g - ref).max()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dims,mode", [((64, 64, 64), 1), ((3, 256, 700), 1), ((700, 224), 1), ((2, 300, 5000), 1)])
def test_gram_split_exact_24bit(P, dims, mode, prec):
    """24-bit data (|x| < 8 on a 2^-20 grid): the three slices represent every
    element exactly and all nine slice products are formed without rounding.
    What rounds is the combination of the orders after each 128-product
    window: the orders >= 2 are added in FP32 (round to nearest, <= 2^-40 of
    the window's largest entry), the rest in double-float and FP64."""
    rng = np.random.default_rng(12)
    x = (rng.integers(-(2 ** 23) + 1, 2 ** 23, size=dims) * 2.0 ** -20).astype(np.float32)
    L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
    g = P.atc_gram(cuda(x), L, n, R, prec).cpu().numpy()
    ref = O.mode_gram(x.astype(np.float64), mode)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dims,mode,r", [((64, 64, 64), 1, 40), ((3, 256, 700), 1, 130), ((700, 224), 1, 16)])
def test_ttm_split_exact_integer(P, dims, mode, r, prec):
    """x on an 8-bit grid and factor entries k/256 with |k| < 256: single
    slices, all partial sums integers below 2^24, so Y must equal the exact
    product rounded once to FP32."""
    rng = np.random.default_rng(13)
    x = (rng.integers(-255, 256, size=dims) * 0.125).astype(np.float32)
    x.flat[0] = 255 * 0.125
    u = rng.integers(-255, 256, size=(dims[mode], r)) / 256.0
    L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
    y = P.atc_ttm(cuda(x), L, n, R, cuda(u), r, expand=False, precision=prec, out_dtype=torch.float32).cpu().numpy()
    ref = O.ttm_project(x.astype(np.float64), u, mode).astype(np.float32)
    assert np.array_equal(y.reshape(ref.shape), ref)


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
    _check_split_against_oracle(P, c, x, 1e-2, ref)


def _principal_angle(u, v):
    qu, _ = np.linalg.qr(u)
    qv, _ = np.linalg.qr(v)
    s = np.linalg.svd(qu.T @ qv, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_pipeline_split_bumps256(P, prec, eps):
    x = synth.gaussian_bumps()
    ref = O.sthosvd(x, eps)
    c = P.atc_compress(cuda(x), eps, precision=prec)
    assert c.ranks() == ref["ranks"], (c.ranks(), ref["ranks"])
    # at 1e-3 every mode's leading eigenvectors come from the subspace iteration
    # (at 1e-4, ranks near 24, a mode may also take the full solver; the ranks are
    # certified either way)
    if eps == 1e-3:
        assert c.stats()["subspace_modes"] == 3
    # a smooth field's cut sits in a fast-falling spectrum: no mode needs four slices
    assert c.stats()["escalated_modes"] == 0
    for m in range(x.ndim):
        u = c.factor(m).cpu().numpy()
        assert np.abs(u.T @ u - np.eye(u.shape[1])).max() <= 1e-12
        # the split Gram matrix is that of X on a 24-bit fixed-point grid, so the
        # last kept directions are fixed only to about (slicing perturbation) /
        # (eigenvalue gap at the cut): measured 4e-5 rad at 1e-3, 6e-4 at 1e-4
        assert _principal_angle(u, ref["factors"][m]) <= 2e-3
    _check_split_against_oracle(P, c, x, eps, ref)


def _check_split_against_oracle(P, c, x, eps, ref):
    """The split path's output against the oracle's on the same input:
    * the ST-HOSVD reconstruction core x_1 U_1 .. x_d U_d (before quantization)
      within 1e-5 ||X|| of the oracle's (the two quantized reconstructions each
      carry their own quantization noise of size ~eps ||X||, so the 1e-5 bar
      applies to the transform; the decoded stream is held to the oracle's
      decoder and to the error bound instead);
    * storage order and the stream header fields (dims, ranks, order, dtype,
      scale exponent k, block size) equal the oracle stream's;
    * the oracle decodes the GPU stream to the GPU's own decompression (1e-9);
    * the achieved error lies in [0.98, 1] * eps."""
    x64 = np.asarray(x, dtype=np.float64)
    nx = np.linalg.norm(x64)
    core = c.core().cpu().numpy()
    fac = [c.factor(m).cpu().numpy() for m in range(x.ndim)]
    xt_gpu = O.reconstruct(core, fac)
    xt_ref = O.reconstruct(ref["core"], ref["factors"])
    assert np.linalg.norm(xt_gpu - xt_ref) <= 1e-5 * nx, np.linalg.norm(xt_gpu - xt_ref) / nx
    st = c.stats()
    assert list(st["storage_order"]) == O.storage_order(ref["ranks"])
    stream = c.stream_bytes()
    s_ref, _ = OP.compress(x, eps)
    hg, hr = OP.parse(stream), OP.parse(s_ref)
    for key in ("dims", "ranks", "perm", "dtype"):
        assert hg[key] == hr[key], (key, hg[key], hr[key])
    qg, qr = OQ.peek(hg["core_stream"]), OQ.peek(hr["core_stream"])
    for key in ("n", "k", "block_size"):
        assert qg[key] == qr[key], (key, qg, qr)
    # dropped factor columns: exactly the slices without a significant coefficient
    # in the GPU's own quantized core (the quantizer is bit-exact on it)
    vec = OP.vectorize_core(core, hg["perm"])
    q, _ = OQ.quantize(vec, qg["k"])
    kept = OP.kept_columns(OP.significant(q, qg["p_star"], qg["i_lead"]), hg["ranks"], hg["perm"])
    for kg, ke in zip(hg["kept"], kept):
        assert np.array_equal(kg, ke)
    xh = P.atc_decompress(stream).cpu().numpy()
    xo = OP.decompress(stream)
    assert np.linalg.norm(xo - xh) <= 1e-9 * nx
    re = np.linalg.norm(x64 - xh) / nx
    assert 0.98 * eps <= re <= eps, re


@pytest.mark.parametrize("prec", [1, 2])
def test_decompress_split_expansion(P, prec):
    """The tensor-core expansion (atc_decompress_ex) reproduces the FP64
    expansion of the same stream to FP32 level (spec bar: 1e-5)."""
    x = synth.lowrank_tucker()
    c = P.atc_compress(cuda(x), 1e-2, precision=prec)
    s = c.stream_bytes()
    x64 = P.atc_decompress(s).cpu().numpy()
    xs = P.atc_decompress(s, out_dtype=torch.float32, precision=prec).cpu().numpy().astype(np.float64)
    xs64 = P.atc_decompress(s, out_dtype=torch.float64, precision=prec).cpu().numpy()
    nx = np.linalg.norm(x)
    assert np.linalg.norm(xs - x64) <= 1e-6 * nx
    assert np.array_equal(xs64, xs)
    re = np.linalg.norm(x - xs) / nx
    assert 0.98e-2 <= re <= 1e-2, re


@pytest.mark.parametrize("eps,prec", [(1e-3, 1), (1e-4, 1), (1e-3, 2)])
def test_certified_tails_match_measured_truncation(P, eps, prec):
    """The split paths certify each mode's tail as trace(G) - sum_{j<r}
    u_j^T G u_j (FP64, G the tensor-core Gram matrix).  Summed over the modes
    this is the ST-HOSVD truncation error of the returned core and factors
    (Theorem 6.4 of the cited ST-HOSVD paper, for any orthonormal factors):
    ||X - core x_i U_i||^2, measured here in FP64 on the host, must agree to
    second order in the 24-bit slicing and the FP32 intermediates."""
    x = synth.gaussian_bumps()
    c = P.atc_compress(cuda(x), eps, precision=prec)
    st = c.stats()
    core = c.core().cpu().numpy()
    t = core
    for i in range(3):
        t = O.ttm_expand(t, c.factor(i).cpu().numpy(), i)
    measured = float(np.sum((x.astype(np.float64) - t) ** 2))
    nx2 = st["norm2"]
    assert abs(st["sse_trunc"] - measured) <= 1e-3 * measured + 1e-11 * nx2, (st["sse_trunc"], measured)
    assert st["sse_trunc"] <= st["target_sse"]


@pytest.mark.parametrize("prec", [1, 2])
def test_gram_converter_kernel_matches_tma_kernel(P, monkeypatch, prec):
    """ATC_GRAM_CONVERT=1 selects the converter-warp Gram (the input sliced by
    warps inside the kernel instead of the separate slicing pass + TMA): on
    24-bit data both are exact to the same FP64 sums, so they agree with each
    other and with the oracle's FP64 Gram."""
    dims = (37, 300, 29)
    rng = np.random.default_rng(41)
    x = (rng.integers(-(2 ** 23) + 1, 2 ** 23, size=dims) * 2.0 ** -20).astype(np.float32)
    out = {}
    for mode in (0, 1, 2):
        L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
        ref = O.mode_gram(x.astype(np.float64), mode)
        for conv in ("1", "0"):
            monkeypatch.setenv("ATC_GRAM_CONVERT", conv)
            g = P.atc_gram(cuda(x), L, n, R, prec).cpu().numpy()
            assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max(), (mode, conv)
            out[(mode, conv)] = g
        assert np.abs(out[(mode, "1")] - out[(mode, "0")]).max() <= 1e-12 * np.abs(ref).max()


def test_split_full_eigensolver_switch(P, monkeypatch):
    """ATC_SUBSPACE=0 sends every mode of a split path through the full
    double-float eigensolver (the fallback of the subspace iteration): the
    ranks still equal the oracle's and the error bound holds."""
    monkeypatch.setenv("ATC_SUBSPACE", "0")
    x = synth.gaussian_bumps(n=128, nbumps=16, seed=31)
    ref = O.sthosvd(x, 1e-3)
    c = P.atc_compress(cuda(x), 1e-3, precision=1)
    assert c.stats()["subspace_modes"] == 0
    assert c.ranks() == ref["ranks"], (c.ranks(), ref["ranks"])
    _check_split_against_oracle(P, c, x, 1e-3, ref)
    monkeypatch.setenv("ATC_SUBSPACE", "1")
    c2 = P.atc_compress(cuda(x), 1e-3, precision=1)
    assert c2.ranks() == ref["ranks"]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("dims,mode", [((6, 200, 70), 1), ((300, 96), 0), ((50, 224), 1)])
def test_gram_wide_32bit(P, dims, mode, prec, dtype):
    """ATC_PREC_WIDE: four 8-bit slices per value (32-bit fixed point below
    max |x|).  On data that 32-bit fixed point holds exactly -- 31-bit integer
    mantissas in FP64, or FP32 values whose magnitudes spread over 2^8 (as in a
    projected tensor) -- the Gram matrix matches the FP64 one to the
    double-float running sums and the dropped products of order >= 5 (~2^-39
    relative), where three slices round the data to 24 bits below max |x|; R = 1
    (the last mode) takes the transposing slicer."""
    rng = np.random.default_rng(51)
    if dtype == np.float64:
        x = rng.integers(-(2 ** 31) + 1, 2 ** 31, size=dims) * 2.0 ** -28
    else:
        e = rng.integers(0, 9, size=dims)
        x = (rng.integers(-(2 ** 23) + 1, 2 ** 23, size=dims) * 2.0 ** (-20 - e)).astype(np.float32)
        x.flat[0] = (2 ** 23 - 1) * 2.0 ** -20
    L = int(np.prod(dims[:mode])); n = dims[mode]; R = int(np.prod(dims[mode + 1:]))
    ref = O.mode_gram(x.astype(np.float64), mode)
    gw = P.atc_gram(cuda(x), L, n, R, prec | P.PREC_WIDE).cpu().numpy()
    g3 = P.atc_gram(cuda(x), L, n, R, prec).cpu().numpy()
    scale = np.abs(ref).max()
    err_w = np.abs(gw - ref).max() / scale
    err_3 = np.abs(g3 - ref).max() / scale
    assert err_w <= 1e-11, err_w
    assert err_w <= 1e-3 * err_3, (err_w, err_3)
    assert np.array_equal(gw, gw.T)


def test_pipeline_split_wide_bumps(P):
    """A whole split compression with four-slice Grams in every mode (ranks,
    error bound and the oracle comparisons as for three slices)."""
    x = synth.gaussian_bumps(n=128, nbumps=16, seed=31)
    ref = O.sthosvd(x, 1e-3)
    c = P.atc_compress(cuda(x), 1e-3, precision=P.PREC_SPLIT_BF16 | P.PREC_WIDE)
    assert c.ranks() == ref["ranks"]
    assert c.stats()["escalated_modes"] == 0
    _check_split_against_oracle(P, c, x, 1e-3, ref)
