"""Host-side checks of the C ABI library (no GPU needed): it builds, loads and
exports every entry point include/atc.h declares; argument validation happens
on the host before any device work."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2107_01384_gb300 as P
    return P.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "atc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(atc_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    import paper_2107_01384_gb300 as P
    assert declared_symbols() == sorted(P.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2107_01384_gb300", "libatc.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(atc_[a-z0-9_]+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_host_validation_rejects_bad_arguments(lib):
    import ctypes as C
    import paper_2107_01384_gb300 as P
    opt = P.Options()
    lib.atc_default_options(C.byref(opt))
    assert abs(opt.rtmss - 0.5) < 1e-15 and opt.block_size == 4096 and opt.precision == 0
    h = C.c_void_p()
    dims = (C.c_int64 * 3)(4, 4, 4)
    # NULL tensor
    assert lib.atc_compress(None, dims, 3, 1, 1e-2, None, C.byref(h)) == -1
    fake = C.c_void_p(0x1000)  # never dereferenced: validation fails first
    assert lib.atc_compress(fake, dims, 9, 1, 1e-2, None, C.byref(h)) == -1
    assert lib.atc_compress(fake, dims, 3, 7, 1e-2, None, C.byref(h)) == -1
    for eps in (0.0, -1.0, 1.5, float("nan")):
        assert lib.atc_compress(fake, dims, 3, 1, eps, None, C.byref(h)) == -1
    bad = (C.c_int64 * 3)(4, 0, 4)
    assert lib.atc_compress(fake, bad, 3, 1, 1e-2, None, C.byref(h)) == -1
    opt.rtmss = 2.0
    assert lib.atc_compress(fake, dims, 3, 1, 1e-2, C.byref(opt), C.byref(h)) == -1
    lib.atc_default_options(C.byref(opt))
    opt.block_size = 100
    assert lib.atc_compress(fake, dims, 3, 1, 1e-2, C.byref(opt), C.byref(h)) == -1
    lib.atc_default_options(C.byref(opt))
    order = (C.c_int * 3)(0, 0, 2)
    opt.mode_order = order
    assert lib.atc_compress(fake, dims, 3, 1, 1e-2, C.byref(opt), C.byref(h)) == -1
    assert b"permutation" in lib.atc_last_error()
    # the no-allocation Gram checks n before forming n * n (2^32 would wrap to 0)
    # and refuses an index range beyond int64, before touching the device
    assert lib.atc_gram_fp64_noalloc(fake, 1, 1, 2 ** 32, 1, fake, None) == -1
    assert b"no-allocation maximum" in lib.atc_last_error()
    assert lib.atc_gram_fp64_noalloc(fake, 1, 2 ** 40, 2, 2 ** 40, fake, None) == -1
    assert b"overflows" in lib.atc_last_error()


def test_stream_header_checks_on_host(lib):
    import ctypes as C
    nd, dt = C.c_int(0), C.c_int(0)
    dims = (C.c_int64 * 8)()
    assert lib.atc_peek_dims(b"XXXX" + b"\0" * 60, 64, C.byref(nd), dims, C.byref(dt)) == -4
    import struct
    hdr = b"ATC1" + struct.pack("<III", 2, 3, 1) + struct.pack("<3Q", 5, 6, 7)
    assert lib.atc_peek_dims(hdr + b"\0" * 64, len(hdr) + 64, C.byref(nd), dims, C.byref(dt)) == 0
    assert nd.value == 3 and list(dims)[:3] == [5, 6, 7] and dt.value == 1
    assert lib.atc_peek_dims(hdr[:20], 20, C.byref(nd), dims, C.byref(dt)) == -4
    # the version-1 layout (all factor columns, no column maps) is not read
    old = b"ATC1" + struct.pack("<III", 1, 3, 1) + struct.pack("<3Q", 5, 6, 7)
    assert lib.atc_peek_dims(old + b"\0" * 64, len(old) + 64, C.byref(nd), dims, C.byref(dt)) == -4


def test_batch_create_rejects_bad_arguments_on_the_host(lib):
    """atc_batch_create validates shapes, dtype and rel_eps before touching the device."""
    import ctypes as C
    h = C.c_void_p()
    dims = (C.c_int64 * 6)(16, 20, 24, 30, 31, 32)
    eps = (C.c_double * 2)(1e-2, 1e-3)
    assert lib.atc_batch_create(0, 3, dims, 1, eps, None, C.byref(h)) == -1
    assert lib.atc_batch_create(2, 9, dims, 1, eps, None, C.byref(h)) == -1
    assert lib.atc_batch_create(2, 3, None, 1, eps, None, C.byref(h)) == -1
    assert lib.atc_batch_create(2, 3, dims, 2, eps, None, C.byref(h)) == -5   # float64: unsupported
    big = (C.c_int64 * 6)(16, 20, 113, 30, 31, 32)
    assert lib.atc_batch_create(2, 3, big, 1, eps, None, C.byref(h)) == -5    # mode > 112
    zero = (C.c_int64 * 6)(16, 0, 24, 30, 31, 32)
    assert lib.atc_batch_create(2, 3, zero, 1, eps, None, C.byref(h)) == -1
    for bad in (0.0, 1.5, float("nan")):
        e2 = (C.c_double * 2)(1e-2, bad)
        assert lib.atc_batch_create(2, 3, dims, 1, e2, None, C.byref(h)) == -1
    assert not h.value
