"""GPU Dslash and operator parity against the FP64 oracle (through the C ABI).

Tolerances (relative L2 over the output field, against the oracle run on the
same unquantised FP64 inputs): FP64 1e-13, FP32 1e-6, FP16 5e-3.  Sizes span
a partial block (4^4), a ragged tail (4x6x8x10: 960 sites per parity, not a
multiple of the 256-thread block) and several full tiles; the full 32^4
workload is checked on sampled output sites.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import TOL_DSLASH, Field, dev, rel_l2, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

DIMS = [(4, 4, 4, 4), (4, 6, 8, 10), (8, 8, 8, 8), (12, 8, 6, 10)]


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("recon", [18, 12])
def test_dslash_all_precisions(dims, recon):
    stag = _stag()
    f = Field.get(dims)
    h = f.handle(recon=recon)
    lat = synth.Lattice(dims)
    for out_parity in (0, 1):
        psi = synth.random_spinor(dims, 7 + out_parity)
        ref = oracle.dslash(f.fat, f.lng, psi, dims, out_parity)
        pd = dev(psi)
        for prec, tol in TOL_DSLASH.items():
            out = torch.empty_like(pd)
            stag.stag_dslash(h, out, pd, out_parity, prec)
            torch.cuda.synchronize()
            err = rel_l2(out.cpu().numpy(), ref)
            assert err < tol, (dims, recon, out_parity, prec, err)
            if prec == "fx16":
                assert err < 5e-4, (dims, recon, out_parity, prec, err)
    assert lat.Vh == h.Vh
    h.free()


@pytest.mark.parametrize("nrhs", [2, 3, 4, 8, 11])
def test_dslash_multiple_rhs(nrhs):
    """N-right-hand-side kernel (groups of 8, 4, 2 plus a single one) in every format."""
    stag = _stag()
    dims = (4, 6, 8, 10)
    f = Field.get(dims)
    h = f.handle(recon=12)
    psi = np.stack([synth.random_spinor(dims, 20 + k) for k in range(nrhs)])
    refs = [oracle.dslash(f.fat, f.lng, psi[k], dims, 1) for k in range(nrhs)]
    for prec, tol in TOL_DSLASH.items():
        out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
        stag.stag_dslash(h, out, dev(psi), 1, prec, nrhs=nrhs)
        got = out.cpu().numpy()
        for k in range(nrhs):
            assert rel_l2(got[k], refs[k]) < tol, (prec, nrhs, k)
    h.free()


@pytest.mark.parametrize("prec,tol", list(TOL_DSLASH.items()))
def test_apply_m(prec, tol):
    stag = _stag()
    dims = (8, 8, 8, 8)
    f = Field.get(dims)
    h = f.handle(recon=12)
    v = synth.random_spinor(dims, 31)
    out = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
    stag.stag_apply_m(h, out, dev(v), 0.1, shift=0.02, prec=prec)
    ref = oracle.apply_m(f.fat, f.lng, v, 0.1, dims, shift=0.02)
    assert rel_l2(out.cpu().numpy(), ref) < tol
    h.free()


def test_free_field_through_gpu():
    """Unit links (eps = 0): the GPU operator reproduces the closed-form eigenvalue."""
    stag = _stag()
    dims = (4, 6, 8, 10)
    fat, lng = synth.gauge_field(dims, 0.0, 1)
    h = stag.stag_load_links(dims, dev(fat), dev(lng), recon_long=12)
    lex = oracle.parity_sites(dims, 0)
    c = oracle.site_coords(dims, lex)
    n = np.array([1, 2, 3, 4])
    p = 2 * np.pi * n / np.array(dims)
    psi = np.exp(1j * (c @ p))[:, None] * np.array([0.3, -0.5j, 0.2 + 0.1j])[None, :]
    lam = 0.01 + np.sum((1.75 * np.sin(p) - np.sin(3 * p) / 24) ** 2)
    for prec, tol in TOL_DSLASH.items():
        out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
        stag.stag_apply_m(h, out, dev(psi), 0.1, prec=prec)
        assert rel_l2(out.cpu().numpy(), lam * psi) < tol
    h.free()


@pytest.mark.parametrize("prec,recon", [("fp64", 18), ("fp32", 12), ("fp16", 12), ("fx16", 12), ("fp32", 18), ("fx16", 18),
                                        ("fx16l", 12)])
def test_dslash_32_4_sampled_sites(prec, recon):
    """Full-size 32^4 workload: sampled output sites vs the oracle site by site."""
    stag = _stag()
    dims = (32, 32, 32, 32)
    f = Field.get(dims)
    h = f.handle(recon=recon, prec_mask=(1 << stag.PREC["fx16" if prec == "fx16l" else prec]))
    psi = synth.random_spinor(dims, 41)
    pd = dev(psi)
    out = torch.empty_like(pd)
    stag.stag_dslash(h, out, pd, 1, prec)
    got = out.cpu().numpy()
    rng = np.random.default_rng(5)
    sites = np.unique(np.concatenate([rng.integers(0, h.Vh, 4000), [0, 1, 15, 16, h.Vh - 1]]))
    ref = oracle.dslash(f.fat, f.lng, psi, dims, 1, out_sites=sites)
    assert rel_l2(got[sites], ref) < TOL_DSLASH[prec]
    h.free()


def test_dslash_32_4_four_rhs_sampled_sites():
    """The headline's operator: four right-hand sides in one FP32 launch (the
    register-capped kernel), 32^4, sampled sites of every vector vs the oracle."""
    stag = _stag()
    dims = (32, 32, 32, 32)
    f = Field.get(dims)
    h = f.handle(recon=12, prec_mask=(1 << stag.PREC["fp32"]))
    psi = np.stack([synth.random_spinor(dims, 60 + k) for k in range(4)])
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    stag.stag_dslash(h, out, dev(psi), 1, "fp32", nrhs=4)
    got = out.cpu().numpy()
    rng = np.random.default_rng(6)
    sites = np.unique(np.concatenate([rng.integers(0, h.Vh, 2000), [0, 1, 15, 16, h.Vh - 1]]))
    for k in range(4):
        ref = oracle.dslash(f.fat, f.lng, psi[k], dims, 1, out_sites=sites)
        assert rel_l2(got[k][sites], ref) < TOL_DSLASH["fp32"], k
    h.free()
