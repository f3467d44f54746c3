"""GPU fermion force through the fat and Naik link construction against the
FP64 oracle: element by element on lattices whose extents keep the one-,
two- and three-hop neighbours distinct (each term type alone and all
together, several weighted solution pairs), the whole chain from thin links
through multi-shift CG and D_oe to the force, gauge covariance at the
benchmark's 32^4, and rejected inputs."""

import numpy as np
import pytest
import torch

import oracle
import oracle.fermion_force as ff
import synth
from gpu_common import dev, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

FULL = (1.0, 0.125, -1.0 / 24.0)


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


def _fields(dims, n, seed):
    xs = np.stack([synth.random_spinor(dims, seed + i) for i in range(n)])
    ys = np.stack([synth.random_spinor(dims, seed + 100 + i) for i in range(n)])
    return xs, ys


@pytest.mark.parametrize(
    "coef", [(1.0, 0.0, 0.0), (0.0, 0.125, 0.0), (0.0, 0.0, -1.0 / 24.0), FULL], ids=["onelink", "staples", "naik", "all"]
)
def test_fermion_force_matches_oracle(coef):
    stag = _stag()
    dims = (6, 8, 6, 10)
    thin = synth.gauge_field(dims, 0.4, 1080, return_thin=True)[2]
    alphas = (0.8, -0.25, 1.5)
    xs, ys = _fields(dims, 3, 1081)
    F = stag.stag_fermion_force(dims, dev(thin), dev(xs), dev(ys), alphas, *coef).cpu().numpy()
    want = ff.fermion_force(thin, list(xs), list(ys), alphas, dims, *coef)
    err = np.abs(F - want).max() / np.abs(want).max()
    print(f"fermion force {coef}: max rel. error {err:.2e}")
    assert err < 1e-13


def test_fermion_force_16_4_many_terms():
    stag = _stag()
    dims = (16, 16, 16, 16)
    thin = synth.gauge_field(dims, 0.3, 1082, return_thin=True)[2]
    n = 12
    alphas = tuple(np.linspace(0.1, 1.2, n))
    xs, ys = _fields(dims, n, 1083)
    F = stag.stag_fermion_force(dims, dev(thin), dev(xs), dev(ys), alphas, *FULL).cpu().numpy()
    want = ff.fermion_force(thin, list(xs), list(ys), alphas, dims, *FULL)
    assert np.abs(F - want).max() < 1e-13 * np.abs(want).max()


def test_fermion_force_from_solutions_end_to_end():
    """Thin links -> GPU links -> multi-shift CG -> D_oe -> force on the GPU,
    against the oracle's own chain (links, CG to 1e-13, D_oe, force)."""
    stag = _stag()
    dims = (6, 6, 6, 8)
    mass, shifts, alphas = 0.3, (0.0, 0.05, 0.4), (0.5, 0.3, 0.2)
    thin = synth.gauge_field(dims, 0.4, 1084, return_thin=True)[2]
    phi = synth.gaussian_source(dims, 1085)
    td = dev(thin)
    fat, lng = stag.stag_build_links(dims, td, c1=FULL[0], c_staple=FULL[1], c3=FULL[2])
    h = stag.stag_load_links(dims, fat, lng, recon_long=18, long_coeff=FULL[2])
    xs = torch.zeros((len(shifts), h.Vh, 3), dtype=torch.complex128, device="cuda")
    infos = stag.stag_multishift_cg(h, list(xs), dev(phi), mass, shifts, tol=1e-12)
    assert all(i["converged"] for i in infos), infos
    ys = torch.empty_like(xs)
    stag.stag_dslash(h, ys, xs, 1, prec="fp64", nrhs=len(shifts))
    F = stag.stag_fermion_force(dims, td, xs, ys, alphas, *FULL).cpu().numpy()
    oxs, oys = ff.solutions(thin, phi, mass, shifts, dims, *FULL)
    want = ff.fermion_force(thin, oxs, oys, alphas, dims, *FULL)
    err = np.abs(F - want).max() / np.abs(want).max()
    print(f"end-to-end fermion force max rel. error {err:.2e}")
    assert err < 1e-8
    h.free()


def test_fermion_force_32_4_gauge_covariance():
    """At the benchmark size: F(gU, gX, gY) = g F(U, X, Y) g^dag link by link."""
    stag = _stag()
    dims = (32, 32, 32, 32)
    thin = synth.gauge_field(dims, 0.3, 1000, return_thin=True)[2]
    alphas = (0.6, 0.4)
    xs, ys = _fields(dims, 2, 1086)
    F1 = stag.stag_fermion_force(dims, dev(thin), dev(xs), dev(ys), alphas, *FULL).cpu().numpy()
    g = synth.random_gauge_transform(dims, 1087)
    thin2 = synth.gauge_transform_links(dims, thin, g)
    del thin
    ev, od = oracle.parity_sites(dims, 0), oracle.parity_sites(dims, 1)
    xs2 = np.stack([np.einsum("nij,nj->ni", g[ev], x) for x in xs])
    ys2 = np.stack([np.einsum("nij,nj->ni", g[od], y) for y in ys])
    F2 = stag.stag_fermion_force(dims, dev(thin2), dev(xs2), dev(ys2), alphas, *FULL).cpu().numpy()
    want = g[:, None] @ F1 @ np.conj(np.swapaxes(g, 1, 2))[:, None]
    assert np.abs(F2 - want).max() < 1e-12 * np.abs(F1).max()


def test_fermion_force_rejects_bad_inputs():
    stag = _stag()
    dims = (4, 4, 4, 4)
    t = torch.zeros((256, 4, 3, 3), dtype=torch.complex128, device="cuda")
    x = torch.zeros((1, 128, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(stag.StagError):
        stag.stag_fermion_force(dims, t, x, x, (1.0,), force=t)  # force overlaps thin
    with pytest.raises(stag.StagError):
        stag.stag_fermion_force(dims, t, x[:0], x[:0], ())  # no terms
    x33 = torch.zeros((33, 128, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(stag.StagError):
        stag.stag_fermion_force(dims, t, x33, x33, (1.0,) * 33)  # more than 32 terms
