"""stag_apply_m_noalloc, the operator entry point that allocates no device
memory (for callers whose device memory belongs to their own allocator, or
whose post-start-up code may not allocate).  Its result must match the
allocating stag_apply_m and the FP64 oracle, call after call, although every
call reuses the same static scratch array; the device's free memory must not
change across its calls; overlapping input and output are refused.
Collected last on purpose: it runs after every other test in a full run, and
also passes alone in a fresh process."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import TOL_DSLASH, Field, dev, rel_l2, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


def _call_noalloc(stag, h, out, inp, mass, shift):
    """Straight through the C ABI: device pointers and the current stream."""
    st = stag._lib.stag_apply_m_noalloc(
        h.ptr,
        ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(inp.data_ptr()),
        ctypes.c_double(mass),
        ctypes.c_double(shift),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
    )
    assert st == stag.STAG_OK, stag.strerror(st)


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (16, 16, 16, 32)])
def test_noalloc_matches_allocating_apply_twice(dims):
    stag = _stag()
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_FP64)
    assert h.Vh <= stag.NOALLOC_MAX_VH
    mass, shift = 0.05, 0.01
    for call, seed in enumerate((61, 62)):
        v = dev(synth.random_spinor(dims, seed))
        ref = torch.empty_like(v)
        stag.stag_apply_m(h, ref, v, mass, shift=shift, prec="fp64")
        got = torch.full_like(v, complex(np.nan, np.nan))
        _call_noalloc(stag, h, got, v, mass, shift)
        torch.cuda.synchronize()
        got_h = got.cpu().numpy()
        err = rel_l2(got_h, ref.cpu().numpy())
        assert err < TOL_DSLASH["fp64"], (dims, call, err)
        err_o = rel_l2(got_h, oracle.apply_m(f.fat, f.lng, synth.random_spinor(dims, seed), mass, dims, shift=shift))
        assert err_o < TOL_DSLASH["fp64"], (dims, call, err_o)
    h.free()


def test_noalloc_leaves_device_memory_unchanged():
    """The defining property: after a first call (which looks up the scratch
    array's address), further calls change the device's free memory by
    nothing at all."""
    stag = _stag()
    dims = (8, 8, 8, 8)
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_FP64)
    v = dev(synth.random_spinor(dims, 63))
    out = torch.empty_like(v)
    _call_noalloc(stag, h, out, v, 0.1, 0.0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _call_noalloc(stag, h, out, v, 0.1, 0.0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    h.free()


def test_noalloc_refuses_overlapping_input_and_output():
    stag = _stag()
    dims = (8, 8, 8, 8)
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_FP64)
    buf = torch.zeros((h.Vh + 1, 3), dtype=torch.complex128, device="cuda")
    for out in (buf[: h.Vh], buf[1:]):
        st = stag._lib.stag_apply_m_noalloc(
            h.ptr, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(buf.data_ptr()), 0.1, 0.0, None
        )
        assert st == stag.STAG_EINVAL
    h.free()


def test_noalloc_rejects_lattice_above_its_limit():
    stag = _stag()
    dims = (16, 16, 16, 34)  # V/2 = 69632 > 65536
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_FP64)
    assert h.Vh > stag.NOALLOC_MAX_VH
    v = torch.zeros((h.Vh, 3), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(v)
    st = stag._lib.stag_apply_m_noalloc(
        h.ptr, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(v.data_ptr()), 0.1, 0.0, None
    )
    assert st == stag.STAG_EINVAL
    h.free()
