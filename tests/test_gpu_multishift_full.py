"""The multi-shift workload at full size: 48^3 x 96, m = 0.005, nine shifts
10^(-4 + k/2), one Gaussian source, FP32 Dslash in the shared Krylov loop and
FP64 refinement, every shifted solution to 1e-10.  The FP64 true residuals
come from the GPU; the oracle recomputes M x site by site on a sample of
2000 even sites for every shift and checks the residual there."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import dev, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_multishift_48c96_mixed32():
    import paper_1712_00143_gb300 as stag

    dims = (48, 48, 48, 96)
    mass = 0.005
    shifts = [10 ** (-4 + k / 2) for k in range(9)]
    fat, lng = synth.gauge_field(dims, 0.3, 1000)
    h = stag.stag_load_links(dims, dev(fat), dev(lng), recon_long=12, prec_mask=(1 << stag.STAG_FP64) | (1 << stag.STAG_FP32))
    b = synth.gaussian_source(dims, 5000)
    bd = dev(b)
    xs = [torch.zeros_like(bd) for _ in shifts]
    infos = stag.stag_multishift_cg(h, xs, bd, mass, shifts, mode="mixed32", tol=1e-10)
    h.free()
    del bd
    rng = np.random.default_rng(11)
    sites = np.unique(rng.integers(0, b.shape[0], 2000))
    for s, x, inf in zip(shifts, xs, infos):
        assert inf["converged"] and inf["true_rel_resid"] <= 1e-10, (s, inf)
        xh = x.cpu().numpy()
        mx = oracle.apply_m_at_sites(fat, lng, xh, mass, dims, sites, shift=s)
        r = b[sites] - mx
        # a sample of the residual field: its size relative to b's on the
        # same sites tracks the global 1e-10 (allow sampling spread)
        assert np.linalg.norm(r) / np.linalg.norm(b[sites]) < 3e-10, (s, inf)
    its = [inf["iters"] for inf in infos]
    assert its[0] == max(its)
