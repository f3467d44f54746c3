"""Writes tests/golden/oracle_fixtures.json: small values computed by the FP64
oracle (only oracle/ and the seeded input generators are called) that the CPU
test test_golden.py recomputes, so that any later change to the oracle's
arithmetic shows up as a diff of this file and needs a stated reason.

The paper prints no worked example (no operator, no solver trace, no force
values), so no fixture here is a value from the paper.

Run from the repository root:  python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import oracle.fermion_force as ff  # noqa: E402
import oracle.gauge_force as gf  # noqa: E402
import oracle.links as olk  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fixtures.json")


def cplx(a):
    a = np.asarray(a).ravel()
    return [[float(v.real), float(v.imag)] for v in a]


def fixtures():
    out = {}
    # Dslash D_oe on 4x6x4x8, seeded links and field: the first 4 odd sites
    dims = (4, 6, 4, 8)
    fat, lng = synth.gauge_field(dims, 0.3, 1090)
    psi = synth.random_spinor(dims, 1091)
    d = oracle.dslash(fat, lng, psi, dims, out_parity=1)
    out["dslash_oe_4x6x4x8"] = {
        "inputs": "synth.gauge_field(dims, 0.3, 1090), synth.random_spinor(dims, 1091)",
        "first_sites": cplx(d[:4]),
        "norm": float(np.linalg.norm(d)),
    }
    # FP64 CG on 4^4, m = 0.1, source 5000: iterations, residual and Lanczos extremes
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, 1007)
    b = synth.gaussian_source(dims, 5000)
    x, info = oracle.cg(fat, lng, b, 0.1, dims, tol=1e-10)
    out["cg_4x4x4x4_m0.1"] = {
        "inputs": "synth.gauge_field(dims, 0.3, 1007), synth.gaussian_source(dims, 5000), mass 0.1, tol 1e-10",
        "iters": int(info["iters"]),
        "x_first_site": cplx(x[0]),
        "ritz_min": float(info["ritz"][0]),
        "ritz_max": float(info["ritz"][-1]),
    }
    # links, gauge force and fermion force on 4x4x4x6 / 6^4: sampled links
    dims = (4, 4, 4, 6)
    thin = synth.gauge_field(dims, 0.4, 1060, return_thin=True)[2]
    F = olk.fat_links(thin, dims)
    L = olk.naik_links(thin, dims)
    G = gf.force(thin, dims, 6.0, *gf.luscher_weisz_coefficients(0.87))
    out["links_and_gauge_force_4x4x4x6"] = {
        "inputs": "thin = synth.gauge_field(dims, 0.4, 1060, return_thin=True)[2]; (1, 1/8, -1/24); beta 6, u0 0.87",
        "fat_site5_mu2": cplx(F[5, 2]),
        "naik_site17_mu3": cplx(L[17, 3]),
        "gauge_force_site33_mu1": cplx(G[33, 1]),
    }
    dims = (6, 6, 6, 6)
    thin = synth.gauge_field(dims, 0.4, 1070, return_thin=True)[2]
    xs = [synth.random_spinor(dims, 1092), synth.random_spinor(dims, 1093)]
    ys = [synth.random_spinor(dims, 1094), synth.random_spinor(dims, 1095)]
    FF = ff.fermion_force(thin, xs, ys, (0.7, -0.2), dims)
    out["fermion_force_6x6x6x6"] = {
        "inputs": "thin = synth.gauge_field(dims, 0.4, 1070, return_thin=True)[2]; X = random_spinor 1092, 1093; "
        "Y = random_spinor 1094, 1095; alpha (0.7, -0.2); (1, 1/8, -1/24)",
        "site7_mu0": cplx(FF[7, 0]),
        "site500_mu3": cplx(FF[500, 3]),
    }
    return out


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(fixtures(), fh, indent=1)
    print("wrote", OUT)
