"""Pins of the fermion-force oracle (CPU): the factor lists rebuild the fat
and Naik links; finite differences of the two-shift pseudofermion action on
single links match the force, for the one-link, staple and Naik terms
separately and together; gauge covariance; planted errors (a dropped
dagger in a staple factor, a flipped sign of the odd-site outer product)
are caught by the finite differences."""

import numpy as np
import pytest
import scipy.linalg

import oracle.fermion_force as ff
import oracle.links as olk
import synth

# extents >= 6 in every direction, so that y + 2 mu and y - 2 mu (and the
# three-hop neighbours) are distinct sites
DIMS = (6, 6, 6, 6)
V = int(np.prod(DIMS))
MASS = 0.5
SHIFTS = (0.0, 0.3)
ALPHAS = (0.7, 0.4)
FULL = (1.0, 0.125, -1.0 / 24.0)


@pytest.fixture(scope="module")
def thin():
    return synth.gauge_field(DIMS, 0.4, 1070, return_thin=True)[2]


@pytest.fixture(scope="module")
def phi():
    return synth.gaussian_source(DIMS, 1071)


def _su3_algebra(rng):
    A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    X = 0.5 * (A - A.conj().T)
    return X - np.trace(X) / 3.0 * np.eye(3)


def test_link_terms_rebuild_the_links():
    dims = (4, 6, 4, 8)
    u = synth.gauge_field(dims, 0.5, 1072, return_thin=True)[2]
    c1, cst, c3 = 0.9, 0.11, -0.05
    terms = ff.link_terms(dims, c1, cst, c3)
    assert [len(terms["fat"][mu]) for mu in range(4)] == [7] * 4  # one link + 3 x 2 staples
    np.testing.assert_allclose(ff.build_from_terms(u, terms["fat"]), olk.fat_links(u, dims, c1, cst), atol=1e-14)
    np.testing.assert_allclose(ff.build_from_terms(u, terms["naik"]), olk.naik_links(u, dims, c3), atol=1e-14)


def _fd_check(u, phi, coef, links, eps=1e-3, rtol=2e-7):
    """Four-point finite differences of S along exp(t X) U on each link of
    `links` against -Re Tr(X F)."""
    xs, ys = ff.solutions(u, phi, MASS, SHIFTS, DIMS, *coef)
    F = ff.fermion_force(u, xs, ys, ALPHAS, DIMS, *coef)
    rng = np.random.default_rng(7)
    out = []
    for site, mu in links:
        X = _su3_algebra(rng)

        def S(t):
            v = u.copy()
            v[site, mu] = scipy.linalg.expm(t * X) @ u[site, mu]
            return ff.action(v, phi, MASS, SHIFTS, ALPHAS, DIMS, *coef)

        fd = (-S(2 * eps) + 8 * S(eps) - 8 * S(-eps) + S(-2 * eps)) / (12 * eps)
        want = -np.real(np.trace(X @ F[site, mu]))
        out.append((fd, want))
        assert abs(fd - want) < rtol * max(1.0, abs(want)) + 1e-9, (site, mu, fd, want)
    return out


# one even and one odd site per case, different directions
LINKS = [(0, 0), (1 + 6 * (2 + 6 * (3 + 6 * 4)), 3), (7 + 36 * 5, 1)]


@pytest.mark.parametrize(
    "coef", [(1.0, 0.0, 0.0), (0.0, 0.125, 0.0), (0.0, 0.0, -1.0 / 24.0), FULL], ids=["onelink", "staples", "naik", "all"]
)
def test_force_is_minus_the_action_derivative(thin, phi, coef):
    pairs = _fd_check(thin, phi, coef, LINKS)
    assert max(abs(w) for _, w in pairs) > 1e-3  # the pin is not vacuous


def test_gauge_covariance(thin):
    rng = np.random.default_rng(3)
    X = [synth.random_spinor(DIMS, 1073), synth.random_spinor(DIMS, 1074)]
    Y = [synth.random_spinor(DIMS, 1075), synth.random_spinor(DIMS, 1076)]
    alphas = (0.6, -0.3)
    F = ff.fermion_force(thin, X, Y, alphas, DIMS, *FULL)
    g = synth.random_gauge_transform(DIMS, 1077)
    u2 = synth.gauge_transform_links(DIMS, thin, g)
    from oracle import parity_sites

    ev, od = parity_sites(DIMS, 0), parity_sites(DIMS, 1)
    X2 = [np.einsum("nij,nj->ni", g[ev], x) for x in X]
    Y2 = [np.einsum("nij,nj->ni", g[od], y) for y in Y]
    F2 = ff.fermion_force(u2, X2, Y2, alphas, DIMS, *FULL)
    want = np.einsum("nij,nmjk,nlk->nmil", g, F, np.conj(g))
    np.testing.assert_allclose(F2, want, atol=1e-12)
    assert rng is not None


def test_planted_dagger_error_is_caught(thin, phi, monkeypatch):
    orig = ff.link_terms

    def broken(dims, c1, c_st, c3):
        t = orig(dims, c1, c_st, c3)
        coef, factors = t["fat"][2][1]  # the first upper staple of F_z
        s, d, _ = factors[2]
        t["fat"][2][1] = (coef, factors[:2] + [(s, d, False)])
        return t

    monkeypatch.setattr(ff, "link_terms", broken)
    with pytest.raises(AssertionError):
        _fd_check(thin, phi, (0.0, 0.125, 0.0), [(0, 2), (36 + 1, 0)])


def test_planted_sign_error_is_caught(thin, phi, monkeypatch):
    orig = ff.outer_products

    def broken(xs, ys, alphas, dims):
        GF, GL = orig(xs, ys, alphas, dims)
        from oracle import parity_sites

        od = parity_sites(dims, 1)
        GF[od] = -GF[od]
        return GF, GL

    monkeypatch.setattr(ff, "outer_products", broken)
    with pytest.raises(AssertionError):
        _fd_check(thin, phi, (1.0, 0.0, 0.0), [(0, 0), (1, 0)])
