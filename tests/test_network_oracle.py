"""Pins of the network oracle (CPU): the backward pass against FP64 finite
differences of the loss, adjointness of the transports, gauge covariance of
the network, and the bfloat16 rounding."""

import numpy as np
import pytest

import oracle
import oracle.network as net
import synth

DIMS = (4, 4, 4, 6)


@pytest.fixture(scope="module")
def setup():
    fat, lng, thin = synth.gauge_field(DIMS, 0.3, 1010, return_thin=True)
    even = oracle.parity_sites(DIMS, 0)
    r = synth.random_spinor(DIMS, 21)
    e = synth.random_spinor(DIMS, 22)
    return fat, thin, even, r, e


def test_transport_adjoints(setup):
    fat, thin, even, r, e = setup
    V = fat.shape[0]
    a = synth.random_spinor(DIMS, 31, full=True).reshape(1, V, 3)
    b = synth.random_spinor(DIMS, 32, full=True).reshape(1, V, 3)
    for d in range(net.NDIR):
        lhs = np.vdot(a, net.transport(fat, b, DIMS, d))
        rhs = np.vdot(net.transport_adjoint(fat, a, DIMS, d), b)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_transports_sum_to_the_fat_part_of_dslash(setup):
    """sum_{d != 0} T_d h restricted to odd sites = D_oe h with the Naik links set to zero."""
    fat, thin, even, r, e = setup
    V = fat.shape[0]
    h = np.zeros((1, V, 3), dtype=np.complex128)
    h[0, even] = r
    tot = sum(net.transport(fat, h, DIMS, d) for d in range(1, net.NDIR))
    odd = oracle.parity_sites(DIMS, 1)
    want = oracle.dslash(fat, np.zeros_like(fat), r, DIMS, out_parity=1)
    assert np.abs(tot[0, odd] - want).max() < 1e-14
    assert np.abs(tot[0, even]).max() == 0.0


@pytest.mark.parametrize("channels", [(1, 2, 1), (1, 3, 2, 1)])
def test_backward_matches_finite_differences(setup, channels):
    fat, thin, even, r, e = setup
    params = net.init_params(channels, 5)
    params = [(W, None if b is None else b + 0.3) for W, b in params]
    L, grads = net.backward(fat, params, r, e, DIMS, even)
    rng = np.random.default_rng(1)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for _ in range(4):
            idx = tuple(rng.integers(0, n) for n in W.shape)
            Wp = W.copy()
            Wp[idx] += h
            Wm = W.copy()
            Wm[idx] -= h
            pp = list(params)
            pp[li] = (Wp, b)
            Lp = net.loss(fat, pp, r, e, DIMS, even)[0]
            pp[li] = (Wm, b)
            Lm = net.loss(fat, pp, r, e, DIMS, even)[0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grads[li][0][idx]) < 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][0][idx])
        if b is not None:
            for c in range(len(b)):
                bp, bm = b.copy(), b.copy()
                bp[c] += h
                bm[c] -= h
                pp = list(params)
                pp[li] = (W, bp)
                Lp = net.loss(fat, pp, r, e, DIMS, even)[0]
                pp[li] = (W, bm)
                Lm = net.loss(fat, pp, r, e, DIMS, even)[0]
                fd = (Lp - Lm) / (2 * h)
                assert abs(fd - grads[li][1][c]) < 1e-6 * max(1.0, abs(fd))


def test_network_is_gauge_covariant(setup):
    fat, thin, even, r, e = setup
    params = net.init_params((1, 4, 4, 1), 7)
    params = [(W, None if b is None else b - 0.2) for W, b in params]
    g = synth.random_gauge_transform(DIMS, 44)
    fat2, _ = synth.links_from_thin(DIMS, synth.gauge_transform_links(DIMS, thin, g))
    gr = np.einsum("nij,nj->ni", g[even], r)
    z1, _ = net.forward(fat, params, r, DIMS, even)
    z2, _ = net.forward(fat2, params, gr, DIMS, even)
    assert np.abs(z2 - np.einsum("nij,nj->ni", g[even], z1)).max() < 1e-12 * np.abs(z1).max()


def test_planted_wrong_adjoint_fails_finite_differences(setup, monkeypatch):
    fat, thin, even, r, e = setup
    params = net.init_params((1, 2, 1), 5)
    monkeypatch.setattr(net, "transport_adjoint", lambda f, g, dims, d: net.transport(f, g, dims, d))
    L, grads = net.backward(fat, params, r, e, DIMS, even)
    W, b = params[0]
    bad = 0
    for idx in [(1, 0, 0), (3, 1, 0), (6, 0, 0)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += 1e-6
        Wm[idx] -= 1e-6
        Lp = net.loss(fat, [(Wp, b)] + params[1:], r, e, DIMS, even)[0]
        Lm = net.loss(fat, [(Wm, b)] + params[1:], r, e, DIMS, even)[0]
        bad += abs((Lp - Lm) / 2e-6 - grads[0][0][idx]) > 1e-4
    assert bad > 0


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: near 1 the spacing is 2^-7
    vals = np.array([1.0, 1 + 2.0**-8, 1 + 3 * 2.0**-8, 1 + 1.5 * 2.0**-8, -3.14159265, 1e-3])
    got = net.bf16_round(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0  # exact tie: to even
    assert got[2] == 1 + 2 * 2.0**-7  # exact tie: to even (upwards here)
    assert got[3] == 1 + 2.0**-7
    assert np.all(np.abs(got - vals) <= np.abs(vals) * 2.0**-8)


MASS = 0.07


@pytest.fixture(scope="module")
def with_long():
    fat, lng = synth.gauge_field(DIMS, 0.3, 1010)
    return fat, lng


@pytest.mark.parametrize("channels", [(1, 2, 1), (1, 3, 2, 1)])
def test_residual_loss_backward_matches_finite_differences(setup, with_long, channels):
    fat, thin, even, r, e = setup
    fat, lng = with_long
    params = net.init_params(channels, 6)
    params = [(W, None if b is None else b + 0.2) for W, b in params]
    L, grads = net.backward_residual(fat, lng, params, r, MASS, DIMS, even)
    rng = np.random.default_rng(3)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        idxs = [tuple(rng.integers(0, n) for n in W.shape) for _ in range(4)]
        for idx in idxs:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params)
            pp[li] = (Wp, b)
            Lp = net.loss_residual(fat, lng, pp, r, MASS, DIMS, even)[0]
            pp[li] = (Wm, b)
            Lm = net.loss_residual(fat, lng, pp, r, MASS, DIMS, even)[0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grads[li][0][idx]) < 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][0][idx])
        if b is not None:
            bp, bm = b.copy(), b.copy()
            bp[0] += h
            bm[0] -= h
            pp = list(params)
            pp[li] = (W, bp)
            Lp = net.loss_residual(fat, lng, pp, r, MASS, DIMS, even)[0]
            pp[li] = (W, bm)
            Lm = net.loss_residual(fat, lng, pp, r, MASS, DIMS, even)[0]
            assert abs((Lp - Lm) / (2 * h) - grads[li][1][0]) < 1e-6 * max(1.0, abs(grads[li][1][0]))


def test_residual_loss_of_a_scaled_identity_is_a_least_squares_fit(setup, with_long):
    """A single linear layer with only the self direction, weight w, gives
    z = w r, so L_r(w) = ||w M r^ - r^||^2 / ||r^||^2: a quadratic in w whose
    minimum sits at w* = Re<M r^, r^> / ||M r^||^2 with value
    1 - Re<M r^, r^>^2 / (||M r^||^2 ||r^||^2), where dL/dw vanishes."""
    fat, thin, even, r, e = setup
    fat, lng = with_long
    rhat = r * np.sqrt(len(even)) / np.linalg.norm(r)
    Mr = oracle.apply_m(fat, lng, rhat, MASS, DIMS)
    a = np.vdot(Mr, rhat).real
    w_star = a / np.linalg.norm(Mr) ** 2
    W = np.zeros((net.NDIR, 1, 1))
    W[0, 0, 0] = w_star
    L, grads = net.backward_residual(fat, lng, [(W, None)], r, MASS, DIMS, even)
    want = 1.0 - a * a / (np.linalg.norm(Mr) ** 2 * np.linalg.norm(rhat) ** 2)
    assert abs(L - want) < 1e-12
    assert abs(grads[0][0][0, 0, 0]) < 1e-10
    # away from w*: the quadratic, exactly
    W[0, 0, 0] = 2.0 * w_star
    L2 = net.loss_residual(fat, lng, [(W, None)], r, MASS, DIMS, even)[0]
    assert abs(L2 - np.linalg.norm(2.0 * w_star * Mr - rhat) ** 2 / np.linalg.norm(rhat) ** 2) < 1e-12


def test_residual_loss_equals_m_weighted_error(setup, with_long):
    """With r = M e the residual loss is ||M (z^ - e^)||^2 / ||M e^||^2."""
    fat, thin, even, r, e = setup
    fat, lng = with_long
    r = oracle.apply_m(fat, lng, e, MASS, DIMS)
    params = net.init_params((1, 2, 1), 8)
    L, cache = net.loss_residual(fat, lng, params, r, MASS, DIMS, even)
    s = cache["scale"]
    zhat = cache["h"][-1][0, even]
    want = np.linalg.norm(oracle.apply_m(fat, lng, zhat - e * s, MASS, DIMS)) ** 2 / np.linalg.norm(r * s) ** 2
    assert abs(L - want) < 1e-11 * max(1.0, want)


@pytest.mark.parametrize("dims", [(8, 6, 8, 10), (4, 4, 4, 6)])
def test_forward_at_sites_equals_the_whole_field_forward(dims):
    """The sampled-site forward (layer k evaluated only on the sites within
    L - k hops of the requested outputs) must reproduce the whole-field
    forward at those sites: on 8x6x8x10 the four-hop neighbourhoods stay
    well inside the lattice, on 4^3x6 they wrap around it."""
    fat, _ = synth.gauge_field(dims, 0.3, 1040)
    even = oracle.parity_sites(dims, 0)
    r = synth.random_spinor(dims, 23)
    params = net.init_params((1, 3, 2, 2, 1), seed=4)
    rng = np.random.default_rng(2)
    params = [(W, None if b is None else rng.normal(0.0, 0.5, b.shape)) for W, b in params]
    z, _ = net.forward(fat, params, r, dims, even)
    sites = np.concatenate([rng.integers(0, len(even), 12), [0, len(even) - 1, 5]])
    zs = net.forward_at_sites(fat, params, r, dims, even, sites)
    assert zs.shape == (len(sites), 3)
    assert np.abs(zs - z[sites]).max() < 1e-13 * np.abs(z).max()
