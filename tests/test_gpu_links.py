"""GPU link construction (fat and Naik links from thin links, FP64) against
the FP64 oracle: small lattices element by element, a ragged extent mix, the
32^4 benchmark lattice on sampled sites, and the solver run on GPU-built
links reaching the oracle's true residual."""

import numpy as np
import pytest
import torch

import oracle
import oracle.links as olk
import synth
from gpu_common import dev, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (8, 6, 4, 10), (8, 8, 8, 8)])
def test_build_links_matches_oracle(dims):
    stag = _stag()
    _, _, thin = synth.gauge_field(dims, 0.3, 1050, return_thin=True)
    fat, lng = stag.stag_build_links(dims, dev(thin))
    torch.cuda.synchronize()
    fo = olk.fat_links(thin, dims)
    lo = olk.naik_links(thin, dims)
    assert np.abs(fat.cpu().numpy() - fo).max() < 1e-14 * np.abs(fo).max()
    assert np.abs(lng.cpu().numpy() - lo).max() < 1e-14 * np.abs(lo).max()


def test_build_links_coefficients():
    """Other coefficients scale the two terms of F and the Naik product as stated."""
    stag = _stag()
    dims = (4, 4, 4, 4)
    _, _, thin = synth.gauge_field(dims, 0.5, 1051, return_thin=True)
    fat, lng = stag.stag_build_links(dims, dev(thin), c1=0.3, c_staple=-0.7, c3=2.5)
    fo = olk.fat_links(thin, dims, c1=0.3, c_st=-0.7)
    lo = olk.naik_links(thin, dims, c3=2.5)
    assert np.abs(fat.cpu().numpy() - fo).max() < 1e-13
    assert np.abs(lng.cpu().numpy() - lo).max() < 1e-13


def test_build_links_rejects_aliasing_and_bad_extents():
    stag = _stag()
    dims = (4, 4, 4, 4)
    t = torch.zeros((256, 4, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(stag.StagError):
        stag.stag_build_links(dims, t, fat=t)
    t5 = torch.zeros((320, 4, 3, 3), dtype=torch.complex128, device="cuda")  # 4 x 4 x 4 x 5: odd extent
    with pytest.raises(stag.StagError):
        stag.stag_build_links((4, 4, 4, 5), t5)


def test_build_links_32_4_sampled():
    """The benchmark lattice: sampled sites against the oracle's definition."""
    stag = _stag()
    dims = (32, 32, 32, 32)
    _, _, thin = synth.gauge_field(dims, 0.3, 1000, return_thin=True)
    fat, lng = stag.stag_build_links(dims, dev(thin))
    fat, lng = fat.cpu().numpy(), lng.cpu().numpy()
    rng = np.random.default_rng(3)
    sites = rng.integers(0, thin.shape[0], 64)
    c = oracle.site_coords(dims, sites)
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))  # noqa: E731
    for mu in range(4):
        want = thin[sites, mu].copy()
        for nu in range(4):
            if nu == mu:
                continue
            xpn = oracle.neighbour_lex(dims, c, nu, 1)
            xpm = oracle.neighbour_lex(dims, c, mu, 1)
            xmn = oracle.neighbour_lex(dims, c, nu, -1)
            xmnpm = oracle.neighbour_lex(dims, oracle.site_coords(dims, xmn), mu, 1)
            want += 0.125 * (thin[sites, nu] @ thin[xpn, mu] @ dag(thin[xpm, nu]))
            want += 0.125 * (dag(thin[xmn, nu]) @ thin[xmn, mu] @ thin[xmnpm, nu])
        assert np.abs(fat[sites, mu] - want).max() < 1e-14
        x1 = oracle.neighbour_lex(dims, c, mu, 1)
        x2 = oracle.neighbour_lex(dims, c, mu, 2)
        wl = -(thin[sites, mu] @ thin[x1, mu] @ thin[x2, mu]) / 24.0
        assert np.abs(lng[sites, mu] - wl).max() < 1e-15


def test_solver_on_gpu_built_links():
    """Links built on the GPU feed stag_load_links and the solver; the FP64
    oracle judges the solution with its own links from the same thin field."""
    stag = _stag()
    dims, mass = (8, 8, 8, 8), 0.1
    _, _, thin = synth.gauge_field(dims, 0.3, 1052, return_thin=True)
    fat, lng = stag.stag_build_links(dims, dev(thin))
    h = stag.stag_load_links(dims, fat, lng, recon_long=12)
    b = synth.gaussian_source(dims, 5000)
    x = torch.zeros((h.Vh, 3), dtype=torch.complex128, device="cuda")
    info = stag.stag_cg(h, x, dev(b), mass, mode="mixedfx16", tol=1e-10)
    fo, lo = olk.fat_links(thin, dims), olk.naik_links(thin, dims)
    res = oracle.true_residual(fo, lo, x.cpu().numpy(), b, mass, dims)
    assert info["converged"] and res <= 1e-10, (info, res)
    h.free()
