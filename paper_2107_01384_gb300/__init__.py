"""Python binding of libatc (include/atc.h): ST-HOSVD + bit-plane core compression on GB300.

Argument marshalling only: every step runs in the CUDA kernels of libatc.so.
PyTorch supplies device memory and the current CUDA stream.  If the library is
missing the import of any entry point fails loudly -- there is no fallback.

Names follow the C ABI: atc_norm2, atc_gram, atc_eig_sym, atc_rank_select,
atc_ttm, atc_quantize_core, atc_dequantize_core, atc_compress, atc_decompress,
atc_peek_dims.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

__all__ = [
    "ATC_F32", "ATC_F64", "PREC_FP64", "PREC_SPLIT_BF16", "PREC_SPLIT_FP16", "PREC_WIDE",
    "RANK_STATIC", "RANK_ADAPTIVE", "AtcError", "lib", "lib_path",
    "atc_norm2", "atc_gram", "atc_gram_fp64_noalloc", "atc_eig_sym", "atc_rank_select", "atc_ttm",
    "atc_quantize_core", "atc_dequantize_core", "atc_compress", "atc_decompress",
    "atc_peek_dims", "Compressed", "EXPORTS", "atc_tucker_expand", "atc_tucker_expand_adjoint",
    "TuckerExpand", "tucker_expand", "Batch", "atc_batch_tune", "kernel_timing", "kernel_times",
]

ATC_F32, ATC_F64 = 1, 2
PREC_FP64, PREC_SPLIT_BF16, PREC_SPLIT_FP16 = 0, 1, 2
PREC_WIDE = 16  # flag: split Grams with four slices (32-bit fixed point)
RANK_STATIC, RANK_ADAPTIVE = 0, 1

HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(HERE, "libatc.so")

# every symbol include/atc.h declares
EXPORTS = [
    "atc_default_options", "atc_compress", "atc_get_ranks", "atc_get_core", "atc_get_factor",
    "atc_get_stream", "atc_get_stats", "atc_free", "atc_peek_dims", "atc_decompress", "atc_decompress_ex",
    "atc_tucker_expand", "atc_tucker_expand_adjoint", "atc_norm2",
    "atc_gram", "atc_eig_sym", "atc_rank_select", "atc_ttm", "atc_quantize_core",
    "atc_dequantize_core", "atc_free_buffer", "atc_release_workspace", "atc_last_error",
    "atc_kernel_launches", "atc_kernel_timing", "atc_kernel_times", "atc_gram_fp64_noalloc",
    "atc_batch_create", "atc_batch_run", "atc_batch_get_ranks", "atc_batch_get_core", "atc_batch_get_factor",
    "atc_batch_get_stats", "atc_batch_get_profile", "atc_batch_last_ms", "atc_batch_tune", "atc_batch_free",
]


class AtcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libatc error {code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("rtmss", C.c_double), ("precision", C.c_int), ("rank_rule", C.c_int),
                ("mode_order", C.POINTER(C.c_int)), ("block_size", C.c_int), ("stream", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("norm2", C.c_double), ("target_sse", C.c_double), ("sse_trunc", C.c_double),
                ("sse_quant_pred", C.c_double), ("order", C.c_int * 8), ("storage_order", C.c_int * 8),
                ("k", C.c_int), ("p_star", C.c_int), ("i_lead", C.c_int64), ("i_trail", C.c_int64),
                ("prio", C.c_int), ("escalated_modes", C.c_int),
                ("ms_norm", C.c_double), ("ms_gram", C.c_double), ("ms_eig", C.c_double),
                ("ms_ttm", C.c_double), ("ms_quant", C.c_double), ("ms_encode", C.c_double),
                ("ms_total", C.c_double), ("subspace_modes", C.c_int), ("block_size", C.c_int)]


_lib = None


def lib():
    """Load libatc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise ImportError(f"libatc.so not found at {lib_path}; run __graft_entry__.build()")
        L = C.CDLL(lib_path)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
        L.atc_last_error.restype = C.c_char_p
        L.atc_default_options.argtypes = [C.POINTER(Options)]
        L.atc_default_options.restype = None
        L.atc_compress.argtypes = [vp, C.POINTER(i64), i32, i32, dbl, C.POINTER(Options), C.POINTER(vp)]
        L.atc_get_ranks.argtypes = [vp, C.POINTER(i64)]
        L.atc_get_core.argtypes = [vp, C.POINTER(vp)]
        L.atc_get_factor.argtypes = [vp, i32, C.POINTER(vp)]
        L.atc_get_stream.argtypes = [vp, C.POINTER(vp), C.POINTER(C.c_size_t)]
        L.atc_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.atc_free.argtypes = [vp]
        L.atc_free.restype = None
        L.atc_peek_dims.argtypes = [C.c_char_p, C.c_size_t, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]
        L.atc_decompress.argtypes = [C.c_char_p, C.c_size_t, vp, i32, vp]
        L.atc_decompress_ex.argtypes = [C.c_char_p, C.c_size_t, vp, i32, C.POINTER(Options)]
        L.atc_tucker_expand.argtypes = [vp, i32, C.POINTER(i64), i32, C.POINTER(vp), C.POINTER(i64), vp, i32,
                                        C.POINTER(Options)]
        L.atc_tucker_expand_adjoint.argtypes = [vp, i32, vp, i32, C.POINTER(i64), i32, C.POINTER(vp), C.POINTER(i64),
                                                vp, C.POINTER(vp), C.POINTER(Options)]
        L.atc_norm2.argtypes = [vp, i64, i32, vp, vp]
        L.atc_gram.argtypes = [vp, i32, i64, i64, i64, i32, vp, vp]
        L.atc_eig_sym.argtypes = [vp, i32, vp, vp, i32, vp]
        L.atc_rank_select.argtypes = [vp, i32, dbl, C.POINTER(i32), C.POINTER(dbl), vp]
        L.atc_ttm.argtypes = [vp, i32, i64, i64, i64, vp, i64, i32, i32, vp, i32, vp]
        L.atc_gram_fp64_noalloc.argtypes = [vp, i32, i64, i64, i64, vp, vp]
        L.atc_quantize_core.argtypes = [vp, i64, dbl, i32, vp, C.POINTER(vp), C.POINTER(C.c_size_t), C.POINTER(i64)]
        L.atc_dequantize_core.argtypes = [C.c_char_p, C.c_size_t, vp, i64, vp]
        L.atc_free_buffer.argtypes = [vp]
        L.atc_free_buffer.restype = None
        L.atc_release_workspace.argtypes = []
        L.atc_kernel_launches.argtypes = []
        L.atc_kernel_launches.restype = C.c_longlong
        L.atc_kernel_timing.argtypes = [i32]
        L.atc_kernel_times.argtypes = [C.c_char_p, C.c_size_t]
        L.atc_batch_create.argtypes = [i32, i32, C.POINTER(i64), i32, C.POINTER(dbl), C.POINTER(Options),
                                       C.POINTER(vp)]
        L.atc_batch_run.argtypes = [vp, C.POINTER(vp), vp]
        L.atc_batch_get_ranks.argtypes = [vp, i32, C.POINTER(i64)]
        L.atc_batch_get_core.argtypes = [vp, i32, C.POINTER(vp)]
        L.atc_batch_get_factor.argtypes = [vp, i32, i32, C.POINTER(vp)]
        L.atc_batch_get_stats.argtypes = [vp, i32, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(i32), C.POINTER(i32)]
        L.atc_batch_get_profile.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(i32)]
        L.atc_batch_last_ms.argtypes = [vp]
        L.atc_batch_last_ms.restype = C.c_float
        L.atc_batch_tune.argtypes = [vp, C.POINTER(i32)]
        L.atc_batch_free.argtypes = [vp]
        L.atc_batch_free.restype = None
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise AtcError(rc, lib().atc_last_error().decode(errors="replace"))


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return ATC_F32
    if t.dtype == torch.float64:
        return ATC_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _dev(t: torch.Tensor):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def atc_norm2(x: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty(1, dtype=torch.float64, device=x.device)
    _check(lib().atc_norm2(_dev(x), x.numel(), _dt(x), _dev(out), _stream(stream)))
    return out


def atc_gram(x: torch.Tensor, L: int, n: int, R: int, precision: int = PREC_FP64, stream=None) -> torch.Tensor:
    assert x.numel() == L * n * R
    g = torch.empty((n, n), dtype=torch.float64, device=x.device)
    _check(lib().atc_gram(_dev(x), _dt(x), L, n, R, precision, _dev(g), _stream(stream)))
    return g


def atc_gram_fp64_noalloc(x: torch.Tensor, L: int, n: int, R: int, out: torch.Tensor, stream=None) -> torch.Tensor:
    """FP64 Gram matrix into the caller's `out` (n x n float64) with no device
    allocation inside the library (see include/atc.h)."""
    assert x.numel() == L * n * R and out.numel() == n * n and out.dtype == torch.float64
    _check(lib().atc_gram_fp64_noalloc(_dev(x), _dt(x), L, n, R, _dev(out), _stream(stream)))
    return out


def atc_eig_sym(g: torch.Tensor, nvec: int, stream=None):
    n = g.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device=g.device)
    v = torch.empty((n, max(nvec, 1)), dtype=torch.float64, device=g.device)
    _check(lib().atc_eig_sym(_dev(g), n, _dev(lam), _dev(v) if nvec > 0 else None, nvec, _stream(stream)))
    return lam, v[:, :nvec]


def atc_rank_select(lam: torch.Tensor, budget: float, stream=None):
    r, disc = C.c_int(0), C.c_double(0.0)
    _check(lib().atc_rank_select(_dev(lam), lam.numel(), float(budget), C.byref(r), C.byref(disc), _stream(stream)))
    return r.value, disc.value


def atc_ttm(x: torch.Tensor, L: int, n: int, R: int, u: torch.Tensor, r: int, expand: bool = False,
            precision: int = PREC_FP64, out_dtype=torch.float64, stream=None) -> torch.Tensor:
    out_mode = n if expand else r
    y = torch.empty(L * out_mode * R, dtype=out_dtype, device=x.device)
    _check(lib().atc_ttm(_dev(x), _dt(x), L, n, R, _dev(u), r, 1 if expand else 0, precision, _dev(y), _dt(y),
                         _stream(stream)))
    return y


def atc_quantize_core(core: torch.Tensor, target_sse: float, block_size: int = 4096, stream=None):
    ptr, nb = C.c_void_p(), C.c_size_t(0)
    info = (C.c_int64 * 5)()
    _check(lib().atc_quantize_core(_dev(core), core.numel(), float(target_sse), block_size, _stream(stream),
                                   C.byref(ptr), C.byref(nb), info))
    data = C.string_at(ptr, nb.value)
    lib().atc_free_buffer(ptr)
    return data, dict(k=info[0], p_star=info[1], prio=info[2], i_lead=info[3], i_trail=info[4])


def atc_dequantize_core(section: bytes, n: int, device="cuda", stream=None) -> torch.Tensor:
    out = torch.empty(n, dtype=torch.float64, device=device)
    _check(lib().atc_dequantize_core(section, len(section), _dev(out), n, _stream(stream)))
    return out


class Compressed:
    """Handle returned by atc_compress (owns the library object)."""

    def __init__(self, handle, ndim, dims):
        self._h = handle
        self.ndim = ndim
        self.dims = list(dims)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().atc_free(self._h)
            self._h = None

    def ranks(self):
        r = (C.c_int64 * self.ndim)()
        _check(lib().atc_get_ranks(self._h, r))
        return list(r)

    def stream_bytes(self) -> bytes:
        p, n = C.c_void_p(), C.c_size_t(0)
        _check(lib().atc_get_stream(self._h, C.byref(p), C.byref(n)))
        return C.string_at(p, n.value)

    def stats(self) -> dict:
        s = Stats()
        _check(lib().atc_get_stats(self._h, C.byref(s)))
        out = {f: getattr(s, f) for f, _ in Stats._fields_}
        out["order"] = list(s.order)[: self.ndim]
        out["storage_order"] = list(s.storage_order)[: self.ndim]
        return out

    def _wrap(self, ptr, shape):
        # copy out of the library-owned device buffer (borrowed view -> clone)
        class _View:
            pass
        v = _View()
        v.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr.value, False),
                                      "version": 3, "strides": None}
        torch.cuda.synchronize()
        return torch.as_tensor(v, device="cuda").clone()

    def core(self) -> torch.Tensor:
        p = C.c_void_p()
        _check(lib().atc_get_core(self._h, C.byref(p)))
        return self._wrap(p, self.ranks())

    def factor(self, mode: int) -> torch.Tensor:
        p = C.c_void_p()
        _check(lib().atc_get_factor(self._h, mode, C.byref(p)))
        return self._wrap(p, [self.dims[mode], self.ranks()[mode]])


def atc_compress(x: torch.Tensor, rel_eps: float, rtmss: float = 0.5, precision: int = PREC_FP64,
                 rank_rule: int = RANK_STATIC, mode_order=None, block_size: int = 4096, stream=None) -> Compressed:
    opt = Options()
    lib().atc_default_options(C.byref(opt))
    opt.rtmss = rtmss
    opt.precision = precision
    opt.rank_rule = rank_rule
    opt.block_size = block_size
    opt.stream = _stream(stream)
    keep = None
    if mode_order is not None:
        keep = (C.c_int * len(mode_order))(*mode_order)
        opt.mode_order = keep
    dims = (C.c_int64 * x.dim())(*x.shape)
    h = C.c_void_p()
    _check(lib().atc_compress(_dev(x), dims, x.dim(), _dt(x), float(rel_eps), C.byref(opt), C.byref(h)))
    return Compressed(h, x.dim(), list(x.shape))


def atc_peek_dims(stream_bytes: bytes):
    nd, dt = C.c_int(0), C.c_int(0)
    dims = (C.c_int64 * 8)()
    _check(lib().atc_peek_dims(stream_bytes, len(stream_bytes), C.byref(nd), dims, C.byref(dt)))
    return list(dims)[: nd.value], dt.value


def atc_decompress(stream_bytes: bytes, out_dtype=torch.float64, device="cuda", stream=None,
                   precision: int = PREC_FP64) -> torch.Tensor:
    """Decode a stream; precision selects the FP64 or the tensor-core expansion."""
    dims, _ = atc_peek_dims(stream_bytes)
    out = torch.empty(dims, dtype=out_dtype, device=device)
    if precision == PREC_FP64:
        _check(lib().atc_decompress(stream_bytes, len(stream_bytes), _dev(out), _dt(out), _stream(stream)))
    else:
        opt = Options()
        lib().atc_default_options(C.byref(opt))
        opt.precision = precision
        opt.stream = _stream(stream)
        _check(lib().atc_decompress_ex(stream_bytes, len(stream_bytes), _dev(out), _dt(out), C.byref(opt)))
    return out


def _opts(precision, stream):
    opt = Options()
    lib().atc_default_options(C.byref(opt))
    opt.precision = precision
    opt.stream = _stream(stream)
    return opt


def atc_tucker_expand(core: torch.Tensor, factors, out_dtype=None, precision: int = PREC_FP64,
                      stream=None) -> torch.Tensor:
    """X_hat = G x_1 U_1 ... x_d U_d on the GPU (factors n_k x r_k, any dtype; used as FP64)."""
    d = core.dim()
    us = [f.to(torch.float64).contiguous() for f in factors]
    dims = [u.shape[0] for u in us]
    out = torch.empty(dims, dtype=out_dtype or core.dtype, device=core.device)
    core = core.contiguous()
    ranks = (C.c_int64 * d)(*core.shape)
    dd = (C.c_int64 * d)(*dims)
    fp = (C.c_void_p * d)(*[u.data_ptr() for u in us])
    opt = _opts(precision, stream)
    _check(lib().atc_tucker_expand(_dev(core), _dt(core), ranks, d, fp, dd, _dev(out), _dt(out), C.byref(opt)))
    return out


def atc_tucker_expand_adjoint(dy: torch.Tensor, core: torch.Tensor, factors, precision: int = PREC_FP64,
                              stream=None):
    """(dL/dG, [dL/dU_k]) in FP64 for the cotangent dy of atc_tucker_expand."""
    d = core.dim()
    us = [f.to(torch.float64).contiguous() for f in factors]
    dims = [u.shape[0] for u in us]
    dy = dy.contiguous()
    core = core.contiguous()
    dcore = torch.empty(core.shape, dtype=torch.float64, device=core.device)
    dfac = [torch.empty(u.shape, dtype=torch.float64, device=core.device) for u in us]
    ranks = (C.c_int64 * d)(*core.shape)
    dd = (C.c_int64 * d)(*dims)
    fp = (C.c_void_p * d)(*[u.data_ptr() for u in us])
    dfp = (C.c_void_p * d)(*[t.data_ptr() for t in dfac])
    opt = _opts(precision, stream)
    _check(lib().atc_tucker_expand_adjoint(_dev(dy), _dt(dy), _dev(core), _dt(core), ranks, d, fp, dd,
                                           _dev(dcore), dfp, C.byref(opt)))
    return dcore, dfac


class TuckerExpand(torch.autograd.Function):
    """Differentiable Tucker expansion: forward atc_tucker_expand, backward the
    hand-written adjoint (gradients to the core and to every factor)."""

    @staticmethod
    def forward(ctx, precision, core, *factors):
        ctx.precision = precision
        ctx.save_for_backward(core, *factors)
        return atc_tucker_expand(core, factors, out_dtype=core.dtype, precision=precision)

    @staticmethod
    def backward(ctx, dy):
        core, *factors = ctx.saved_tensors
        dcore, dfac = atc_tucker_expand_adjoint(dy, core, factors, precision=ctx.precision)
        return (None, dcore.to(core.dtype)) + tuple(g.to(f.dtype) for g, f in zip(dfac, factors))


def tucker_expand(core: torch.Tensor, factors, precision: int = PREC_FP64) -> torch.Tensor:
    return TuckerExpand.apply(precision, core, *factors)



def _borrowed(ptr, shape):
    """Copy of a library-owned FP64 device buffer as a torch tensor."""
    class _View:
        pass
    v = _View()
    v.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": "<f8",
                                  "data": (ptr.value, False), "version": 3, "strides": None}
    return torch.as_tensor(v, device="cuda").clone()


class Batch:
    """Batched ST-HOSVD plan (atc_batch_*): many float32 tensors of one order,
    uneven shapes and per-tensor rel_eps, in one persistent graph-replayed launch."""

    def __init__(self, shapes, rel_eps, rtmss: float = 0.5, rank_rule: int = RANK_STATIC, mode_order=None,
                 stream=None):
        shapes = [tuple(int(v) for v in sh) for sh in shapes]
        if not shapes:
            raise ValueError("empty batch")
        d = len(shapes[0])
        if any(len(sh) != d for sh in shapes):
            raise ValueError("all tensors of a batch must have the same order")
        if len(rel_eps) != len(shapes):
            raise ValueError("one rel_eps per tensor")
        self.shapes, self.ndim, self.count = shapes, d, len(shapes)
        opt = Options()
        lib().atc_default_options(C.byref(opt))
        opt.rtmss = rtmss
        opt.rank_rule = rank_rule
        opt.stream = _stream(stream)
        self._order = None
        if mode_order is not None:
            self._order = (C.c_int * d)(*mode_order)
            opt.mode_order = self._order
        dims = (C.c_int64 * (d * self.count))(*[v for sh in shapes for v in sh])
        eps = (C.c_double * self.count)(*[float(e) for e in rel_eps])
        h = C.c_void_p()
        _check(lib().atc_batch_create(self.count, d, dims, ATC_F32, eps, C.byref(opt), C.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().atc_batch_free(self._h)
            self._h = None

    def run(self, tensors, stream=None) -> float:
        """Compress the device tensors (float32, the planned shapes); returns the device ms."""
        if len(tensors) != self.count:
            raise ValueError("one tensor per planned shape")
        for t, sh in zip(tensors, self.shapes):
            if t.dtype != torch.float32 or tuple(t.shape) != sh:
                raise ValueError(f"expected a float32 tensor of shape {sh}")
        ptrs = (C.c_void_p * self.count)(*[_dev(t).value for t in tensors])
        _check(lib().atc_batch_run(self._h, ptrs, _stream(stream)))
        return float(lib().atc_batch_last_ms(self._h))

    def ranks(self, i: int):
        r = (C.c_int64 * self.ndim)()
        _check(lib().atc_batch_get_ranks(self._h, i, r))
        return list(r)

    def stats(self, i: int) -> dict:
        n2, sse = C.c_double(0), C.c_double(0)
        sw = (C.c_int * self.ndim)()
        st = C.c_int(0)
        _check(lib().atc_batch_get_stats(self._h, i, C.byref(n2), C.byref(sse), sw, C.byref(st)))
        return dict(norm2=n2.value, sse_trunc=sse.value, sweeps=list(sw), status=st.value)

    def profile(self, i: int) -> dict:
        """SM cycles per phase (gram, jacobi, rank, ttm) and rotating Jacobi rounds per mode of tensor i."""
        cyc = (C.c_int64 * 4)()
        rounds = (C.c_int * self.ndim)()
        _check(lib().atc_batch_get_profile(self._h, i, cyc, rounds))
        return dict(gram=cyc[0], jacobi=cyc[1], rank=cyc[2], ttm=cyc[3], rounds=list(rounds))

    def core(self, i: int) -> torch.Tensor:
        p = C.c_void_p()
        _check(lib().atc_batch_get_core(self._h, i, C.byref(p)))
        return _borrowed(p, self.ranks(i))

    def factor(self, i: int, mode: int) -> torch.Tensor:
        p = C.c_void_p()
        _check(lib().atc_batch_get_factor(self._h, i, mode, C.byref(p)))
        return _borrowed(p, [self.shapes[i][mode], self.ranks(i)[mode]])


def atc_batch_tune(stream=None):
    """Measure the batched Gram tile table now; returns the tile edge per mode length."""
    tab = (C.c_int * 113)()
    _check(lib().atc_batch_tune(_stream(stream), tab))
    return list(tab)


def kernel_timing(enable: bool) -> None:
    """Start (True) or stop (False) the library's kernel timer (include/atc.h)."""
    _check(lib().atc_kernel_timing(1 if enable else 0))


def kernel_times() -> dict:
    """{kernel name: dict(launches, ms, bytes, flops, issued)} of the current
    timing window (totals over its launches; see include/atc.h)."""
    buf = C.create_string_buffer(1 << 16)
    _check(lib().atc_kernel_times(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms, by, fl, iss = line.split("|")
        out[name] = dict(launches=int(cnt), ms=float(ms), bytes=float(by), flops=float(fl), issued=float(iss))
    return out
