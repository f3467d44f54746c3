"""Pins of the gauge-force oracle (CPU): loop and staple counts, unit links,
finite differences of the action along su(3) directions on single links,
gauge covariance, and a planted sign error caught by the finite
differences."""

import numpy as np
import pytest
import scipy.linalg

import oracle
import oracle.gauge_force as gf
import synth

DIMS = (4, 4, 4, 6)
V = int(np.prod(DIMS))
COEF = gf.luscher_weisz_coefficients(0.87)
BETA = 6.0


@pytest.fixture(scope="module")
def thin():
    return synth.gauge_field(DIMS, 0.4, 1060, return_thin=True)[2]


def test_loop_and_staple_counts():
    shapes = gf.loop_shapes()
    assert [len(shapes[k]) for k in ("pl", "rt", "pg")] == [6, 12, 16]  # geometric loops per site
    st = gf.staple_paths()
    for mu in range(4):
        assert [len(st[k][mu]) for k in ("pl", "rt", "pg")] == [6, 18, 24]
        assert all(len(s) == 3 for s in st["pl"][mu])
        assert all(len(s) == 5 for s in st["rt"][mu] + st["pg"][mu])


def test_unit_links():
    u = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    u[:] = np.eye(3)
    assert abs(gf.action(u, DIMS, BETA, *COEF)) < 1e-12
    assert np.abs(gf.force(u, DIMS, BETA, *COEF)).max() < 1e-14


def _su3_algebra(rng):
    A = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    X = 0.5 * (A - A.conj().T)
    return X - np.trace(X) / 3.0 * np.eye(3)


@pytest.mark.parametrize("coef", [COEF, (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)])
def test_force_is_minus_the_action_derivative(thin, coef):
    F = gf.force(thin, DIMS, BETA, *coef)
    rng = np.random.default_rng(5)
    eps = 1e-5
    for site, mu in [(0, 0), (37, 1), (200, 2), (V - 1, 3)]:
        X = _su3_algebra(rng)
        up, um = thin.copy(), thin.copy()
        up[site, mu] = scipy.linalg.expm(eps * X) @ thin[site, mu]
        um[site, mu] = scipy.linalg.expm(-eps * X) @ thin[site, mu]
        fd = (gf.action(up, DIMS, BETA, *coef) - gf.action(um, DIMS, BETA, *coef)) / (2 * eps)
        want = -np.real(np.trace(X @ F[site, mu]))
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want)), (site, mu, fd, want)


def test_force_is_traceless_antihermitian_and_gauge_covariant(thin):
    F = gf.force(thin, DIMS, BETA, *COEF)
    assert np.abs(F + np.conj(np.swapaxes(F, -1, -2))).max() < 1e-13
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13
    g = synth.random_gauge_transform(DIMS, 43)
    F2 = gf.force(synth.gauge_transform_links(DIMS, thin, g), DIMS, BETA, *COEF)
    want = g[:, None] @ F @ np.conj(np.swapaxes(g, -1, -2))[:, None]
    assert np.abs(F2 - want).max() < 1e-12


def test_planted_sign_error_fails_finite_differences(thin, monkeypatch):
    orig = gf.traceless_antihermitian
    monkeypatch.setattr(gf, "traceless_antihermitian", lambda M: -orig(M) if M.ndim == 3 else orig(M))
    F = gf.force(thin, DIMS, BETA, *COEF)
    monkeypatch.setattr(gf, "traceless_antihermitian", orig)
    rng = np.random.default_rng(6)
    X = _su3_algebra(rng)
    eps = 1e-5
    up, um = thin.copy(), thin.copy()
    up[5, 1] = scipy.linalg.expm(eps * X) @ thin[5, 1]
    um[5, 1] = scipy.linalg.expm(-eps * X) @ thin[5, 1]
    fd = (gf.action(up, DIMS, BETA, *COEF) - gf.action(um, DIMS, BETA, *COEF)) / (2 * eps)
    assert abs(fd + np.real(np.trace(X @ F[5, 1]))) > 1e-3 * abs(fd)
