"""GPU Symanzik one-loop gauge force against the FP64 oracle: small lattices
element by element for each loop type and the combined action, a ragged
extent mix, and the 24^4 benchmark lattice on sampled links checked with
the oracle's own staple walk."""

import numpy as np
import pytest
import torch

import oracle
import oracle.gauge_force as gf
import synth
from gpu_common import dev, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

BETA = 6.0
COEF = gf.luscher_weisz_coefficients(0.87)


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


@pytest.mark.parametrize("coef", [COEF, (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)])
def test_gauge_force_matches_oracle(coef):
    stag = _stag()
    dims = (4, 4, 4, 6)
    thin = synth.gauge_field(dims, 0.4, 1060, return_thin=True)[2]
    F = stag.stag_gauge_force(dims, dev(thin), BETA, *coef)
    want = gf.force(thin, dims, BETA, *coef)
    assert np.abs(F.cpu().numpy() - want).max() < 1e-13 * max(1.0, np.abs(want).max())


def test_gauge_force_ragged_extents():
    stag = _stag()
    dims = (6, 4, 8, 4)
    thin = synth.gauge_field(dims, 0.3, 1061, return_thin=True)[2]
    F = stag.stag_gauge_force(dims, dev(thin), BETA, *COEF)
    want = gf.force(thin, dims, BETA, *COEF)
    assert np.abs(F.cpu().numpy() - want).max() < 1e-13 * np.abs(want).max()


def test_gauge_force_24_4_sampled():
    stag = _stag()
    dims = (24, 24, 24, 24)
    thin = synth.gauge_field(dims, 0.3, 1000, return_thin=True)[2]
    F = stag.stag_gauge_force(dims, dev(thin), BETA, *COEF).cpu().numpy()
    rng = np.random.default_rng(4)
    sites = rng.integers(0, thin.shape[0], 16)
    paths = gf.staple_paths()
    coef = dict(zip(("pl", "rt", "pg"), COEF))
    c = oracle.site_coords(dims, sites)
    for mu in range(4):
        x_pmu = oracle.neighbour_lex(dims, c, mu, 1)
        sig = np.zeros((len(sites), 3, 3), dtype=np.complex128)
        for kind in ("pl", "rt", "pg"):
            for steps in paths[kind][mu]:
                sig += coef[kind] * gf._path_product(thin, dims, x_pmu, steps)
        want = BETA / 3.0 * gf.traceless_antihermitian(thin[sites, mu] @ sig)
        assert np.abs(F[sites, mu] - want).max() < 1e-13 * np.abs(want).max()


def test_gauge_force_rejects_overlap():
    stag = _stag()
    t = torch.zeros((256, 4, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(stag.StagError):
        stag.stag_gauge_force((4, 4, 4, 4), t, BETA, *COEF, force=t)
