"""Pins of the link-construction oracle (CPU): the unit-link closed form, a
single non-trivial link inserted at the sites the definition names (as W or
W^dag), and gauge covariance of fat and Naik links."""

import numpy as np
import pytest

import oracle
import oracle.links as olk
import synth

DIMS = (4, 6, 4, 8)
V = int(np.prod(DIMS))


def _unit():
    u = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    u[:] = np.eye(3)
    return u


def _lex(x, y, z, t):
    Lx, Ly, Lz, Lt = DIMS
    return (x % Lx) + Lx * ((y % Ly) + Ly * ((z % Lz) + Lz * (t % Lt)))


def _su3(seed):
    return synth.random_su3(1, 0.7, seed, 0).numpy()[0]


def test_unit_links_closed_form():
    u = _unit()
    fat = olk.fat_links(u, DIMS, c1=1.0, c_st=0.125)
    lng = olk.naik_links(u, DIMS, c3=-1.0 / 24.0)
    assert np.abs(fat - 1.75 * np.eye(3)).max() < 1e-15
    assert np.abs(lng + np.eye(3) / 24.0).max() < 1e-16


@pytest.mark.parametrize("nu", [0, 1, 3])
def test_single_link_enters_where_the_definition_says(nu):
    """All links 1 except U_nu(y) = W.  F_mu(x) for mu != nu picks W in the
    upper staple at x = y and in the lower staple at x = y + nu - mu, W^dag in
    the upper staple at x = y - mu and in the lower staple at x = y + nu;
    F_nu(y -+ rho) (rho != nu) picks W as the middle factor of its upper /
    lower staple; F_nu(y) = c1 W + 6 c_st; the Naik links of direction nu at
    y, y - nu, y - 2 nu are c3 W; every other link keeps its unit value."""
    c1, cst, c3 = 1.0, 0.125, -1.0 / 24.0
    y = (1, 2, 3, 5)
    W = _su3(77 + nu)
    u = _unit()
    iy = _lex(*y)
    u[iy, nu] = W
    fat = olk.fat_links(u, DIMS, c1, cst)
    lng = olk.naik_links(u, DIMS, c3)
    I = np.eye(3, dtype=np.complex128)
    base = (c1 + 6 * cst) * I
    want_f = np.broadcast_to(base, (V, 4, 3, 3)).copy()
    want_l = np.broadcast_to(c3 * I, (V, 4, 3, 3)).copy()
    e = [np.eye(4, dtype=int)[m] for m in range(4)]
    ya = np.array(y)
    for mu in range(4):
        if mu == nu:
            continue
        for shift, M in ((0 * e[mu], W), (e[nu] - e[mu], W), (-e[mu], W.conj().T), (e[nu], W.conj().T)):
            want_f[_lex(*(ya + shift)), mu] += cst * (M - I)
    for rho in range(4):  # W as the middle factor of the nu-direction staples at y -+ rho
        if rho != nu:
            want_f[_lex(*(ya - e[rho])), nu] += cst * (W - I)
            want_f[_lex(*(ya + e[rho])), nu] += cst * (W - I)
    want_f[iy, nu] = c1 * W + 6 * cst * I
    for k in range(3):
        want_l[_lex(*(ya - k * e[nu])), nu] = c3 * W
    assert np.abs(fat - want_f).max() < 1e-14
    assert np.abs(lng - want_l).max() < 1e-15


def test_gauge_covariance():
    _, _, thin = synth.gauge_field(DIMS, 0.3, 1040, return_thin=True)
    g = synth.random_gauge_transform(DIMS, 41)
    thin2 = synth.gauge_transform_links(DIMS, thin, g)
    fat, fat2 = olk.fat_links(thin, DIMS), olk.fat_links(thin2, DIMS)
    lng, lng2 = olk.naik_links(thin, DIMS), olk.naik_links(thin2, DIMS)
    c = oracle.site_coords(DIMS, np.arange(V))
    for mu in range(4):
        x1 = oracle.neighbour_lex(DIMS, c, mu, 1)
        x3 = oracle.neighbour_lex(DIMS, c, mu, 3)
        wf = g @ fat[:, mu] @ np.conj(np.swapaxes(g[x1], -1, -2))
        wl = g @ lng[:, mu] @ np.conj(np.swapaxes(g[x3], -1, -2))
        assert np.abs(fat2[:, mu] - wf).max() < 1e-13
        assert np.abs(lng2[:, mu] - wl).max() < 1e-14


def test_planted_wrong_staple_order_breaks_covariance(monkeypatch):
    """A transposed lower staple (U_nu(x-nu+mu) ... at the wrong end) is not
    gauge covariant: the covariance pin catches it."""
    _, _, thin = synth.gauge_field(DIMS, 0.3, 1041, return_thin=True)
    g = synth.random_gauge_transform(DIMS, 42)
    thin2 = synth.gauge_transform_links(DIMS, thin, g)

    def bad_fat(t, dims, c1=1.0, c_st=0.125):
        out = olk.fat_links(t, dims, c1, c_st)
        c = oracle.site_coords(dims, np.arange(t.shape[0]))
        x = oracle.neighbour_lex(dims, c, 1, -1)
        out[:, 0] += c_st * (t[x, 0] @ t[x, 1] - np.conj(np.swapaxes(t[x, 1], -1, -2)) @ t[x, 0])
        return out

    fat, fat2 = bad_fat(thin, DIMS), bad_fat(thin2, DIMS)
    c = oracle.site_coords(DIMS, np.arange(V))
    x1 = oracle.neighbour_lex(DIMS, c, 0, 1)
    wf = g @ fat[:, 0] @ np.conj(np.swapaxes(g[x1], -1, -2))
    assert np.abs(fat2[:, 0] - wf).max() > 1e-6
