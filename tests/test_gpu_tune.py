"""The N-right-hand-side kernels' launch variants and their autotuner on the
GPU.  A variant placed in the tuner's cache under a lattice's key is the one
that lattice's groups run with, so every variant is forced in turn: each must
reproduce the oracle's Dslash (plain kernel, FP32 and 16-bit fixed point) and
drive a batched solve to the oracle's 1e-10 residual (epilogue kernel); the
tuner, left to itself, picks a compiled variant and reports its time."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import TOL_DSLASH, Field, dev, oracle_true_residual, rel_l2, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

DIMS = (4, 6, 8, 10)  # 960 sites per parity: a ragged last block for every split


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


# (threads per site, min blocks per SM) of variants 0..5
VARIANTS = [(1, 1), (1, 6), (2, 4), (2, 6), (4, 4), (4, 6)]


@pytest.mark.parametrize("prec", ["fp32", "fx16", "fx16l"])
@pytest.mark.parametrize("nrhs", [2, 4, 8])
def test_every_variant_matches_the_oracle(prec, nrhs):
    stag = _stag()
    f = Field.get(DIMS)
    psi = np.stack([synth.random_spinor(DIMS, 300 + k) for k in range(nrhs)])
    refs = [oracle.dslash(f.fat, f.lng, psi[k], DIMS, 1) for k in range(nrhs)]
    key = stag.stag_tune_key("dslash_mrhs", prec, 6, nrhs, DIMS)
    seen = set()
    try:
        for v in range(len(VARIANTS)):
            stag.stag_tune_cache_clear()
            stag.stag_tune_cache_put(key, v, 1.0)
            # the fx16l operator reads the 16-bit fixed-point link copy
            h = f.handle(recon=12, prec_mask=1 << stag.PREC["fx16" if prec == "fx16l" else prec])
            out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
            stag.stag_dslash(h, out, dev(psi), 1, prec, nrhs=nrhs)
            got = out.cpu().numpy()
            for k in range(nrhs):
                assert rel_l2(got[k], refs[k]) < TOL_DSLASH[prec], (prec, nrhs, v, k)
            sp, minb, us = stag.stag_tuned_mrhs(h, prec, nrhs)
            seen.add((sp, minb))
            h.free()
    finally:
        stag.stag_tune_cache_clear()
    # FP32 vectors build every split that divides N (the default always)
    if prec in ("fp32", "fx16l"):
        assert {sp for sp, _ in seen} == {s for s in (1, 2, 4) if nrhs % s == 0}, seen


@pytest.mark.parametrize("v", range(6))
def test_batched_solve_with_each_variant(v):
    """The epilogue kernel Ap = m^2 p - D_eo t of every variant inside the
    batched solve: four systems, mixed32, oracle residual over the whole field."""
    stag = _stag()
    dims, mass = (8, 8, 8, 8), 0.05
    f = Field.get(dims)
    b = np.stack([synth.gaussian_source(dims, 5400 + k) for k in range(4)])
    key = stag.stag_tune_key("dslash_mrhs", "fp32", 6, 4, dims)
    key_epi = stag.stag_tune_key("dslash_mrhs_epi", "fp32", 6, 4, dims)
    try:
        stag.stag_tune_cache_clear()
        stag.stag_tune_cache_put(key, v, 1.0)
        stag.stag_tune_cache_put(key_epi, v, 1.0)
        h = f.handle(recon=12)
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        infos = stag.stag_batch_solve([(h, x, dev(b), 4, mass)], mode="mixed32", tol=1e-10)
        assert stag.stag_tuned_mrhs(h, "fp32", 4, epilogue=True)[:2] == VARIANTS[v]
        assert stag.stag_tuned_mrhs_variant(h, "fp32", 4, epilogue=True) == v
        assert stag.stag_tuned_mrhs_variant(h, "fp32", 4) == v
        xh = x.cpu().numpy()
        for i in range(4):
            res = oracle_true_residual(f.fat, f.lng, xh[i], b[i], mass, dims)
            assert infos[i]["converged"] and res <= 1e-10, (v, i, infos[i], res)
        h.free()
    finally:
        stag.stag_tune_cache_clear()


def test_tuner_picks_and_remembers():
    """Without a cached entry the first group times the compiled variants,
    keeps one and stores it under the lattice's key; a second handle of the
    same extents reuses it."""
    stag = _stag()
    dims = (8, 8, 8, 8)
    f = Field.get(dims)
    key = stag.stag_tune_key("dslash_mrhs", "fp32", 6, 4, dims)
    key_epi = stag.stag_tune_key("dslash_mrhs_epi", "fp32", 6, 4, dims)
    stag.stag_tune_cache_clear()
    try:
        h = f.handle(recon=12, prec_mask=1 << stag.STAG_FP32)
        psi = dev(np.stack([synth.random_spinor(dims, 310 + k) for k in range(4)]))
        out = torch.empty_like(psi)
        stag.stag_dslash(h, out, psi, 1, "fp32", nrhs=4)
        sp, minb, us = stag.stag_tuned_mrhs(h, "fp32", 4)
        v, us_cached = stag.stag_tune_cache_get(key)
        assert v >= 0 and VARIANTS[v] == (sp, minb) and us > 0 and us_cached == pytest.approx(us, rel=1e-6)
        # the epilogue form is tuned on its own and cached under its own key
        spe, minbe, use = stag.stag_tuned_mrhs(h, "fp32", 4, epilogue=True)
        ve, use_cached = stag.stag_tune_cache_get(key_epi)
        assert ve >= 0 and VARIANTS[ve] == (spe, minbe) and use > 0 and use_cached == pytest.approx(use, rel=1e-6)
        h2 = f.handle(recon=12, prec_mask=1 << stag.STAG_FP32)
        stag.stag_dslash(h2, out, psi, 1, "fp32", nrhs=4)
        assert stag.stag_tuned_mrhs(h2, "fp32", 4)[:2] == (sp, minb)
        h.free()
        h2.free()
    finally:
        stag.stag_tune_cache_clear()
