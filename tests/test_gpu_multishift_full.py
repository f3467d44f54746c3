"""The multi-shift workload at full size: 48^3 x 96, m = 0.005, nine shifts
10^(-4 + k/2), one Gaussian source, FP32 Dslash in the shared Krylov loop and
FP64-class refinement, every shifted solution to 1e-10.  The oracle
recomputes the residual over the whole field for the smallest and the
largest shift (the hardest and the easiest system), and on a sample of 2000
even sites for every shift."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import dev, oracle_true_residual, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_multishift_48c96_mixed32():
    import paper_1712_00143_gb300 as stag

    dims = (48, 48, 48, 96)
    mass = 0.005
    shifts = [10 ** (-4 + k / 2) for k in range(9)]
    fat, lng = synth.gauge_field(dims, 0.3, 1000)
    h = stag.stag_load_links(dims, dev(fat), dev(lng), recon_long=12,
                             prec_mask=(1 << stag.STAG_FP64) | (1 << stag.STAG_FP32) | (1 << stag.STAG_DF64))
    b = synth.gaussian_source(dims, 5000)
    bd = dev(b)
    xs = [torch.zeros_like(bd) for _ in shifts]
    infos = stag.stag_multishift_cg(h, xs, bd, mass, shifts, mode="mixed32", tol=1e-10)
    h.free()
    del bd
    rng = np.random.default_rng(11)
    sites = np.unique(rng.integers(0, b.shape[0], 2000))
    for k, (s, x, inf) in enumerate(zip(shifts, xs, infos)):
        assert inf["converged"] and inf["true_rel_resid"] <= 1e-10, (s, inf)
        xh = x.cpu().numpy()
        if k in (0, len(shifts) - 1):
            res = oracle_true_residual(fat, lng, xh, b, mass, dims, shift=s)
            print(f"shift {s:.1e}: oracle whole-field residual {res:.3e} (library {inf['true_rel_resid']:.3e})")
            assert res <= 1e-10, (s, res)
        mx = oracle.apply_m_at_sites(fat, lng, xh, mass, dims, sites, shift=s)
        r = b[sites] - mx
        # a sample of the residual field: its size relative to b's on the
        # same sites tracks the global 1e-10 (allow sampling spread)
        assert np.linalg.norm(r) / np.linalg.norm(b[sites]) < 3e-10, (s, inf)
    its = [inf["iters"] for inf in infos]
    assert its[0] == max(its)
