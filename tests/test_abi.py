"""The C ABI library: builds, loads, exports every declared entry point, and
rejects bad arguments before touching the GPU (CPU only)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stag.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(stag_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("stag_load_links", "stag_dslash", "stag_cg", "stag_multishift_cg", "stag_apply_m"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol(lib):
    import paper_1712_00143_gb300 as stag

    assert sorted(stag.EXPORTS) == declared_functions()


def test_invalid_arguments_rejected_without_gpu(lib):
    import paper_1712_00143_gb300 as stag

    L = stag._lib
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(8, 8, 8, 8)
    assert L.stag_load_links(ctypes.byref(h), dims, None, None, None, None) == stag.STAG_EINVAL
    odd = (ctypes.c_int * 4)(8, 7, 8, 8)
    one = ctypes.c_void_p(1)
    assert L.stag_load_links(ctypes.byref(h), odd, one, one, None, None) == stag.STAG_EINVAL
    small = (ctypes.c_int * 4)(8, 2, 8, 8)
    assert L.stag_load_links(ctypes.byref(h), small, one, one, None, None) == stag.STAG_EINVAL
    bad = stag.LinkOpts(13, -1 / 24, 0)
    assert L.stag_load_links(ctypes.byref(h), dims, one, one, ctypes.byref(bad), None) == stag.STAG_EINVAL
    assert L.stag_dslash(None, one, one, 0, 0, 1, None) == stag.STAG_EINVAL
    assert L.stag_cg(None, one, one, 0.1, None, None, None) == stag.STAG_EINVAL
    assert L.stag_multishift_cg(None, None, one, 0.1, None, 0, None, None, None) == stag.STAG_EINVAL
    assert L.stag_free_lattice(None) == stag.STAG_EINVAL
    # the FP64 routines around the solver refuse bad arguments before any CUDA call
    two = ctypes.c_void_p(1 << 40)
    three = ctypes.c_void_p(1 << 41)
    alpha = (ctypes.c_double * 33)(*([1.0] * 33))
    assert L.stag_build_links(dims, None, one, two, 1.0, 0.125, -1 / 24, None) == stag.STAG_EINVAL
    assert L.stag_build_links(odd, one, two, three, 1.0, 0.125, -1 / 24, None) == stag.STAG_EINVAL
    assert L.stag_build_links(dims, one, one, two, 1.0, 0.125, -1 / 24, None) == stag.STAG_EINVAL  # fat == thin
    assert L.stag_gauge_force(dims, None, one, 6.0, 1.0, 0.0, 0.0, None) == stag.STAG_EINVAL
    assert L.stag_gauge_force(small, one, two, 6.0, 1.0, 0.0, 0.0, None) == stag.STAG_EINVAL
    assert L.stag_gauge_force(dims, one, one, 6.0, 1.0, 0.0, 0.0, None) == stag.STAG_EINVAL  # force == thin
    ff = L.stag_fermion_force
    assert ff(dims, one, 0, two, three, alpha, 1.0, 0.125, -1 / 24, ctypes.c_void_p(1 << 42), None) == stag.STAG_EINVAL
    assert ff(dims, one, 33, two, three, alpha, 1.0, 0.125, -1 / 24, ctypes.c_void_p(1 << 42), None) == stag.STAG_EINVAL
    assert ff(dims, one, 1, two, three, None, 1.0, 0.125, -1 / 24, ctypes.c_void_p(1 << 42), None) == stag.STAG_EINVAL
    assert ff(odd, one, 1, two, three, alpha, 1.0, 0.125, -1 / 24, ctypes.c_void_p(1 << 42), None) == stag.STAG_EINVAL
    assert ff(dims, one, 1, two, three, alpha, 1.0, 0.125, -1 / 24, one, None) == stag.STAG_EINVAL  # force == thin
    assert ff(dims, one, 1, two, three, alpha, 1.0, 0.125, -1 / 24, two, None) == stag.STAG_EINVAL  # force == x
    assert stag.strerror(stag.STAG_ENOTCONV).startswith("solver did not converge")


def test_default_params():
    import paper_1712_00143_gb300 as stag

    p = stag.default_params()
    assert p.tol == 1e-10 and p.mode == stag.STAG_MIXED32 and abs(p.delta - 0.1) < 1e-15
    q = stag.default_params(mode="mixed16", tol=1e-8)
    assert q.mode == stag.STAG_MIXED16 and q.tol == 1e-8
