"""The learned preconditioner on the GPU: forward and gradient against the
FP64 network oracle, gauge covariance, training that lowers the loss, and
flexible CG with the network reaching 1e-10 (with and without the fallback);
a trained network takes fewer iterations than the untrained one."""

import numpy as np
import pytest
import torch

import oracle
import oracle.network as onet
import synth
from gpu_common import Field, dev, rel_l2, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

CH = (1, 16, 16, 16, 1)


def _stag():
    import paper_1712_00143_gb300 as stag

    return stag


def _oracle_params(flat, channels):
    """Flat parameter array (library layout) -> oracle (W, b) list."""
    out, off = [], 0
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        W = flat[off : off + 9 * co * ci].astype(np.float64).reshape(9, co, ci)
        off += 9 * co * ci
        b = None
        if l < len(channels) - 2:
            b = flat[off : off + co].astype(np.float64)
            off += co
        out.append((W, b))
    return out


def _flat_grads(grads):
    parts = []
    for dW, db in grads:
        parts.append(dW.ravel())
        if db is not None:
            parts.append(db.ravel())
    return np.concatenate(parts)


def _net_with_biases(stag, seed=3):
    """A fresh network with its gate biases moved off zero, so that the
    gate's gradient is exercised."""
    net = stag.stag_net_create(CH, seed=seed)
    p = stag.stag_net_get_params(net)
    rng = np.random.default_rng(0)
    off = 0
    for l in range(len(CH) - 1):
        off += 9 * CH[l] * CH[l + 1]
        if l < len(CH) - 2:
            p[off : off + CH[l + 1]] = rng.normal(0.0, 0.5, CH[l + 1])
            off += CH[l + 1]
    stag.stag_net_set_params(net, p)
    return net


# 4^3 x 6: 192 sites per parity, three whole 64-site tensor-core tiles;
# 6^4: 648 sites per parity, ten tiles and a ragged one of 8 sites
@pytest.fixture(scope="module", params=[(4, 4, 4, 6), (6, 6, 6, 6)], ids=["4x4x4x6", "6x6x6x6"])
def small(request):
    stag = _stag()
    dims = request.param
    fat, lng, thin = synth.gauge_field(dims, 0.3, 1020, return_thin=True)
    h = stag.stag_load_links(dims, dev(fat), dev(lng), recon_long=12)
    net = _net_with_biases(stag)
    yield dims, fat, lng, thin, h, net
    net.free()
    h.free()


def test_tensor_core_selftest():
    """One tile of tcgen05 products (values exact in bfloat16 and FP32)
    against the CUDA cores: the descriptors, the accumulation over nine
    steps and the tensor-memory read-back must reproduce the sums exactly."""
    assert _stag().stag_tc_selftest() == 0.0


def test_forward_matches_oracle(small):
    """The 16 -> 16 layers mix channels on the tensor cores from bfloat16
    hi + lo parts of the FP32 transports (16 significant bits, error <= 2^-18
    of each value), the other layers in FP32: 5e-5 relative L2 over four
    layers."""
    stag = _stag()
    dims, fat, lng, thin, h, net = small
    r = synth.random_spinor(dims, 51)
    z = torch.empty((h.Vh, 3), dtype=torch.complex128, device="cuda")
    stag.stag_net_apply(net, h, z, dev(r))
    params = _oracle_params(stag.stag_net_get_params(net, rounded=True), CH)
    zo, _ = onet.forward(fat, params, r, dims, oracle.parity_sites(dims, 0))
    err = rel_l2(z.cpu().numpy(), zo)
    print(f"network forward rel. L2 error vs FP64 oracle: {err:.2e}")
    assert err < 5e-5


def test_forward_32_4_sampled_sites():
    """The full-size forward (32^4, 1-16-16-16-1, 8192 tensor-core tiles):
    the oracle evaluates the network on sampled output sites only, layer by
    layer on their four-hop neighbourhoods (oracle.network.forward_at_sites)."""
    stag = _stag()
    dims = (32, 32, 32, 32)
    f = Field.get(dims)
    h = f.handle(recon=12, prec_mask=1 << stag.STAG_FP32)
    net = _net_with_biases(stag)
    r = synth.random_spinor(dims, 55)
    z = torch.empty((h.Vh, 3), dtype=torch.complex128, device="cuda")
    stag.stag_net_apply(net, h, z, dev(r))
    params = _oracle_params(stag.stag_net_get_params(net, rounded=True), CH)
    rng = np.random.default_rng(12)
    sites = np.unique(np.concatenate([rng.integers(0, h.Vh, 300), [0, 63, 64, h.Vh - 1]]))
    zo = onet.forward_at_sites(f.fat, params, r, dims, oracle.parity_sites(dims, 0), sites)
    err = rel_l2(z.cpu().numpy()[sites], zo)
    print(f"32^4 network forward on {len(sites)} sampled sites: rel. L2 error {err:.2e}")
    assert err < 5e-5
    net.free()
    h.free()


@pytest.mark.parametrize("kind", ["error", "residual"])
def test_gradient_matches_oracle(small, kind):
    stag = _stag()
    dims, fat, lng, thin, h, net = small
    mass = 0.05
    r = synth.random_spinor(dims, 52)
    e = synth.random_spinor(dims, 53)
    loss, g = stag.stag_net_loss_grad(net, h, dev(r), dev(e), loss=kind, mass=mass)
    params = _oracle_params(stag.stag_net_get_params(net, rounded=True), CH)
    even = oracle.parity_sites(dims, 0)
    if kind == "error":
        lo, go = onet.backward(fat, params, r, e, dims, even)
    else:
        lo, go = onet.backward_residual(fat, lng, params, r, mass, dims, even)
    go = _flat_grads(go)
    print(f"{kind} loss rel. error {abs(loss - lo) / abs(lo):.2e}, gradient {np.linalg.norm(g - go) / np.linalg.norm(go):.2e}")
    assert abs(loss - lo) < 1e-5 * abs(lo)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-4


def test_network_gauge_covariance_on_gpu(small):
    stag = _stag()
    dims, fat, lng, thin, h, net = small
    g = synth.random_gauge_transform(dims, 61)
    fat2, lng2 = synth.links_from_thin(dims, synth.gauge_transform_links(dims, thin, g))
    h2 = stag.stag_load_links(dims, dev(fat2), dev(lng2), recon_long=12)
    even = oracle.parity_sites(dims, 0)
    r = synth.random_spinor(dims, 54)
    z1 = torch.empty((h.Vh, 3), dtype=torch.complex128, device="cuda")
    z2 = torch.empty_like(z1)
    stag.stag_net_apply(net, h, z1, dev(r))
    stag.stag_net_apply(net, h2, z2, dev(np.einsum("nij,nj->ni", g[even], r)))
    want = np.einsum("nij,nj->ni", g[even], z1.cpu().numpy())
    assert rel_l2(z2.cpu().numpy(), want) < 1e-5
    h2.free()


def test_fcg_with_untrained_network_tracks_cg():
    """The freshly created network is close to the identity, so flexible CG
    with it must behave like CG: same solution, similar iteration count."""
    stag = _stag()
    dims, mass = (8, 8, 8, 8), 0.05
    f = Field.get(dims)
    h = f.handle(recon=12)
    net = stag.stag_net_create(CH, seed=11)
    b = synth.gaussian_source(dims, 9200)
    bd = dev(b)
    x = torch.zeros_like(bd)
    info = stag.stag_cg(h, x, bd, mass, mode="learned", precond=net, tol=1e-10)
    x2 = torch.zeros_like(bd)
    ref = stag.stag_cg(h, x2, bd, mass, mode="mixedfx16", tol=1e-10)
    res = oracle.true_residual(f.fat, f.lng, x.cpu().numpy(), b, mass, dims)
    assert info["converged"] and res <= 1e-10 and info["precond_fallback"] == 0, (info, res)
    assert info["iters"] <= 1.3 * ref["iters"] + 8, (info["iters"], ref["iters"])
    net.free()
    h.free()


@pytest.fixture(scope="module")
def trained():
    """A network trained on pairs from two 8^4 fields (m = 0.05)."""
    stag = _stag()
    from paper_1712_00143_gb300.learned import make_pairs

    dims, mass = (8, 8, 8, 8), 0.05
    handles, pairs = [], []
    for j in range(2):
        fat, lng = synth.gauge_field(dims, 0.3, 1030 + j)
        h = stag.stag_load_links(dims, dev(fat), dev(lng), recon_long=12)
        handles.append(h)
        srcs = [dev(synth.gaussian_source(dims, 7000 + 10 * j + s)) for s in range(2)]
        pairs += make_pairs(h, srcs, mass, iters=[1, 3, 6, 10, 15, 22, 30, 40])
    net = stag.stag_net_create(CH, seed=5)
    losses = stag.stag_net_train(net, pairs, epochs=16, batch=4, lr=2e-3, seed=2, loss="residual", mass=mass)
    yield dims, mass, net, losses, len(pairs)
    net.free()
    for h in handles:
        h.free()


def test_training_lowers_the_loss(trained):
    """The residual-space loss ||M N(r) - r||^2 / ||r||^2 starts far above 1
    (the near-identity network returns about r, and M is not near the
    identity) and must fall well below its start and below 1."""
    dims, mass, net, losses, npairs = trained
    first = losses[:npairs].mean()
    last = losses[-npairs:].mean()
    assert np.all(np.isfinite(losses))
    print(f"residual loss: first epoch {first:.4f}, last epoch {last:.4f}")
    assert last < 0.5 * first and last < 1.0, (first, last)


def test_learned_fcg_converges_and_gains(trained):
    stag = _stag()
    dims, mass, net, losses, npairs = trained
    fat, lng = synth.gauge_field(dims, 0.3, 2000)  # held-out field
    h = stag.stag_load_links(dims, dev(fat), dev(lng), recon_long=12)
    b = synth.gaussian_source(dims, 9000)
    bd = dev(b)
    x = torch.zeros_like(bd)
    info = stag.stag_cg(h, x, bd, mass, mode="learned", precond=net, tol=1e-10)
    res = oracle.true_residual(fat, lng, x.cpu().numpy(), b, mass, dims)
    assert info["converged"] and res <= 1e-10 and info["precond_fallback"] == 0, (info, res)
    # the same solver with the untrained network, and CG without a network,
    # both need more iterations
    raw = stag.stag_net_create(CH, seed=5)
    x2 = torch.zeros_like(bd)
    info_raw = stag.stag_cg(h, x2, bd, mass, mode="learned", precond=raw, tol=1e-10)
    assert info_raw["converged"]
    x3 = torch.zeros_like(bd)
    info_cg = stag.stag_cg(h, x3, bd, mass, mode="mixed32", tol=1e-10)
    print(f"learned FCG iterations: trained {info['iters']}, untrained {info_raw['iters']}, CG {info_cg['iters']}")
    assert info["iters"] < info_raw["iters"]
    assert info["iters"] < 0.9 * info_cg["iters"]
    raw.free()
    h.free()


def test_learned_fallback_on_a_useless_network():
    """A network with all-zero output weights returns z = 0: FCG breaks down
    at once and the mixed-CG fallback must still solve the system."""
    stag = _stag()
    dims, mass = (8, 8, 8, 8), 0.1
    f = Field.get(dims)
    h = f.handle(recon=12)
    net = stag.stag_net_create(CH, seed=9)
    p = stag.stag_net_get_params(net)
    p[:] = 0.0
    stag.stag_net_set_params(net, p)
    b = synth.gaussian_source(dims, 9100)
    x = torch.zeros((h.Vh, 3), dtype=torch.complex128, device="cuda")
    info = stag.stag_cg(h, x, dev(b), mass, mode="learned", precond=net, tol=1e-10)
    res = oracle.true_residual(f.fat, f.lng, x.cpu().numpy(), b, mass, dims)
    assert info["precond_fallback"] == 1 and info["converged"] and res <= 1e-10
    net.free()
    h.free()
