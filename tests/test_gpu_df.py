"""The FP64-class double-float operator (STAG_DF64) against the FP64 oracle.

The mixed-precision solvers recompute their true residual b - M y with this
operator (links and vectors as hi + lo float pairs, products and sums by
error-free transformations on the FP32 pipes), so it is held to the FP64
bound, 1e-13 relative L2 over the output field, on the same lattices as the
other formats (a partial block, a ragged tail, several tiles), for one to
eight right-hand sides (launches of up to four), both parities, the operator
with a shift, and the headline's 32^4 lattice on sampled sites.  Solves with
double-float reliable updates must reach the oracle's 1e-10 whole-field
residual and take the same iterations as with FP64 updates."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import TOL_DSLASH_DF, Field, dev, oracle_true_residual, rel_l2, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

DIMS = [(4, 4, 4, 4), (4, 6, 8, 10), (8, 8, 8, 8), (12, 8, 6, 10)]


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


@pytest.mark.parametrize("dims", DIMS)
def test_df_dslash_and_operator(dims):
    stag = _stag()
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_DF64)
    for out_parity in (0, 1):
        psi = synth.random_spinor(dims, 17 + out_parity)
        ref = oracle.dslash(f.fat, f.lng, psi, dims, out_parity)
        out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
        stag.stag_dslash(h, out, dev(psi), out_parity, "df64")
        err = rel_l2(out.cpu().numpy(), ref)
        print(f"{dims} parity {out_parity}: DF64 Dslash rel. L2 error {err:.2e}")
        assert err < TOL_DSLASH_DF, (dims, out_parity, err)
    v = synth.random_spinor(dims, 19)
    out = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
    stag.stag_apply_m(h, out, dev(v), 0.01, shift=0.003, prec="df64")
    ref = oracle.apply_m(f.fat, f.lng, v, 0.01, dims, shift=0.003)
    err = rel_l2(out.cpu().numpy(), ref)
    print(f"{dims}: DF64 operator rel. L2 error {err:.2e}")
    assert err < TOL_DSLASH_DF, (dims, err)
    h.free()


@pytest.mark.parametrize("nrhs", [2, 3, 4, 5, 8])
def test_df_dslash_multiple_rhs(nrhs):
    """Up to four right-hand sides per launch; five and eight take two launches."""
    stag = _stag()
    dims = (4, 6, 8, 10)
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_DF64)
    psi = np.stack([synth.random_spinor(dims, 120 + k) for k in range(nrhs)])
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    stag.stag_dslash(h, out, dev(psi), 1, "df64", nrhs=nrhs)
    got = out.cpu().numpy()
    for k in range(nrhs):
        assert rel_l2(got[k], oracle.dslash(f.fat, f.lng, psi[k], dims, 1)) < TOL_DSLASH_DF, (nrhs, k)
    h.free()


def test_df_dslash_32_4_four_rhs_sampled_sites():
    """The reliable update's shape in the headline: 32^4, four right-hand
    sides in one launch, sampled output sites of every vector."""
    stag = _stag()
    dims = (32, 32, 32, 32)
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_DF64)
    psi = np.stack([synth.random_spinor(dims, 130 + k) for k in range(4)])
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    stag.stag_dslash(h, out, dev(psi), 1, "df64", nrhs=4)
    got = out.cpu().numpy()
    rng = np.random.default_rng(9)
    sites = np.unique(np.concatenate([rng.integers(0, h.Vh, 2000), [0, 1, 15, 16, h.Vh - 1]]))
    for k in range(4):
        ref = oracle.dslash(f.fat, f.lng, psi[k], dims, 1, out_sites=sites)
        assert rel_l2(got[k][sites], ref) < TOL_DSLASH_DF, k
    h.free()


@pytest.mark.parametrize("scale", [1e-15, 1e15])
def test_df_keeps_its_accuracy_across_exponents(scale):
    """The same field scaled by 1e-15 and 1e15: the exact FP64 -> hi + lo
    split of the input, the double-float arithmetic and the widening of the
    output keep the FP64 bound far from the unit exponent (the lo parts stay
    normal floats down to |value| of about 2^-75)."""
    stag = _stag()
    dims = (4, 6, 8, 10)
    f = Field.get(dims)
    h = f.handle(prec_mask=1 << stag.STAG_DF64)
    v = synth.random_spinor(dims, 3) * scale
    out = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
    stag.stag_apply_m(h, out, dev(v), 0.05, prec="df64")
    err = rel_l2(out.cpu().numpy(), oracle.apply_m(f.fat, f.lng, v, 0.05, dims))
    print(f"scale {scale:.0e}: DF64 operator rel. L2 error {err:.2e}")
    assert err < TOL_DSLASH_DF, (scale, err)
    h.free()


@pytest.mark.parametrize("mode", ["mixed32", "mixedfx16"])
def test_solve_with_df_reliable_updates(mode):
    """The same single-RHS solve with FP64 and with double-float reliable
    updates: both reach the oracle's whole-field 1e-10, with the same
    iteration count to within one check interval."""
    stag = _stag()
    dims, mass = (8, 8, 8, 8), 0.02
    f = Field.get(dims)
    b = synth.gaussian_source(dims, 5100)
    infos = {}
    for name, mask in (("fp64", 0b01111), ("df64", 0b11111)):
        h = f.handle(recon=12, prec_mask=mask)
        x = torch.zeros((h.Vh, 3), dtype=torch.complex128, device="cuda")
        infos[name] = stag.stag_cg(h, x, dev(b), mass, mode=mode, tol=1e-10)
        res = oracle_true_residual(f.fat, f.lng, x.cpu().numpy(), b, mass, dims)
        print(f"{mode} with {name} reliable updates: {infos[name]['iters']} iterations, "
              f"{infos[name]['reliable_updates']} updates, oracle residual {res:.2e}")
        assert infos[name]["converged"] and res <= 1e-10, (name, infos[name], res)
        assert abs(infos[name]["true_rel_resid"] - res) < 1e-3 * res + 1e-14
        h.free()
    assert abs(infos["df64"]["iters"] - infos["fp64"]["iters"]) <= 16


def test_batched_solve_with_df_reliable_updates():
    """Four systems batched (one group): double-float updates against FP64
    updates, every solution judged by the oracle's whole-field residual."""
    stag = _stag()
    dims, mass = (8, 8, 8, 8), 0.02
    f = Field.get(dims)
    b = np.stack([synth.gaussian_source(dims, 5200 + k) for k in range(4)])
    iters = {}
    for name, mask in (("fp64", 0b01111), ("df64", 0b11111)):
        h = f.handle(recon=12, prec_mask=mask)
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        infos = stag.stag_batch_solve([(h, x, dev(b), 4, mass)], mode="mixed32", tol=1e-10)
        xh = x.cpu().numpy()
        for i in range(4):
            res = oracle_true_residual(f.fat, f.lng, xh[i], b[i], mass, dims)
            assert infos[i]["converged"] and res <= 1e-10, (name, i, infos[i], res)
        iters[name] = [i["iters"] for i in infos]
        h.free()
    assert all(abs(a - c) <= 16 for a, c in zip(iters["df64"], iters["fp64"])), iters
