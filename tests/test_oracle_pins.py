"""Pins of the FP64 oracle against facts fixed by mathematics (CPU only).

The paper prints no worked example (Sec. 4 reports only performance), so
the oracle is pinned by closed forms, invariants, special cases and
library routines, chosen so that a plausible slip in the oracle (a dropped
hop, a wrong sign, phase or index, a missing dagger) fails one of them.
The last tests plant such slips into the oracle and check that a pin fails.
"""

import numpy as np
import pytest

import oracle
import oracle.staggered as ost
import synth

C1_ASQTAD, C3_ASQTAD = 9.0 / 8.0, -1.0 / 24.0


def _unit_links(dims, c1, c3):
    V = int(np.prod(dims))
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3))
    return c1 * eye.copy(), c3 * eye.copy()


def _even_plane_wave(dims, n, colour):
    """e^{i p.x} colour on even sites, p_mu = 2 pi n_mu / L_mu."""
    lex = ost.parity_sites(dims, 0)
    c = ost.site_coords(dims, lex)
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    return np.exp(1j * (c @ p))[:, None] * np.asarray(colour)[None, :], p


def _free_eigenvalue(p, c1, c3):
    return float(np.sum((c1 * np.sin(p) + c3 * np.sin(3 * p)) ** 2))


# --------------------------------------------------------------- pin helpers


def free_field_error(dims, c1, c3, mass, momenta, fat=None, lng=None):
    """max over momenta of |M psi - (m^2 + lambda(p)) psi| / |psi| on plane waves."""
    if fat is None:
        fat, lng = _unit_links(dims, c1, c3)
    colour = np.array([0.3 + 0.1j, -0.7j, 0.5])
    worst = 0.0
    for n in momenta:
        psi, p = _even_plane_wave(dims, n, colour)
        lam = mass * mass + _free_eigenvalue(p, c1, c3)
        got = oracle.apply_m(fat, lng, psi, mass, dims)
        worst = max(worst, np.linalg.norm(got - lam * psi) / np.linalg.norm(psi))
    return worst


def antihermiticity_error(dims, fat, lng, seed=11):
    """| <u, D_eo v> + <D_oe u, v> | / (|u||v|) for random u (even), v (odd)."""
    u = synth.random_spinor(dims, seed)
    v = synth.random_spinor(dims, seed + 1)
    a = np.vdot(u, oracle.dslash(fat, lng, v, dims, out_parity=0))
    b = np.vdot(oracle.dslash(fat, lng, u, dims, out_parity=1), v)
    return abs(a + b) / (np.linalg.norm(u) * np.linalg.norm(v))


def covariance_error(dims, eps, seed, out_parity):
    """|| D'(G psi) - G (D psi) || / || D psi || with U' = G U G^dag(x+mu)."""
    fat, lng, thin = synth.gauge_field(dims, eps, seed, return_thin=True)
    g = synth.random_gauge_transform(dims, seed + 7)
    fat2, lng2 = synth.links_from_thin(dims, synth.gauge_transform_links(dims, thin, g))
    psi = synth.random_spinor(dims, seed + 3)
    in_sites = ost.parity_sites(dims, 1 - out_parity)
    out_sites = ost.parity_sites(dims, out_parity)
    gpsi = np.einsum("nij,nj->ni", g[in_sites], psi)
    lhs = oracle.dslash(fat2, lng2, gpsi, dims, out_parity)
    rhs = np.einsum("nij,nj->ni", g[out_sites], oracle.dslash(fat, lng, psi, dims, out_parity))
    return np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs)


MOMENTA_4 = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 1, 0, 0), (1, 2, 3, 1), (3, 1, 2, 2)]
MOMENTA_ASYM = [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 2, 3, 4), (3, 5, 7, 9), (2, 4, 1, 6)]


# --------------------------------------------------------------- link recipe


def test_links_eps_zero_special_case():
    """eps = 0: U = 1, so F = (1 + 6/8) 1 = 7/4 1 and L = -1/24 1 exactly."""
    dims = (4, 4, 4, 6)
    fat, lng, thin = synth.gauge_field(dims, 0.0, 1000, return_thin=True)
    assert np.abs(thin - np.eye(3)).max() < 1e-15
    assert np.abs(fat - 1.75 * np.eye(3)).max() < 1e-15
    assert np.abs(lng + np.eye(3) / 24.0).max() < 1e-15


def test_thin_links_are_su3():
    dims = (4, 4, 6, 4)
    _, _, thin = synth.gauge_field(dims, 0.3, 1001, return_thin=True)
    u = thin.reshape(-1, 3, 3)
    assert np.abs(u @ np.conj(np.swapaxes(u, 1, 2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-14
    # and not trivially close to the identity: eps = 0.3 moves them visibly
    assert np.abs(u - np.eye(3)).max() > 0.1


def test_link_recipe_gauge_covariance():
    """F'(x) = G(x) F(x) G(x+mu)^dag and L'(x) = G(x) L(x) G(x+3mu)^dag."""
    dims = (4, 4, 4, 6)
    fat, lng, thin = synth.gauge_field(dims, 0.3, 1002, return_thin=True)
    g = synth.random_gauge_transform(dims, 99)
    fat2, lng2 = synth.links_from_thin(dims, synth.gauge_transform_links(dims, thin, g))
    c = ost.site_coords(dims, np.arange(int(np.prod(dims))))
    for mu in range(4):
        n1 = ost.neighbour_lex(dims, c, mu, 1)
        n3 = ost.neighbour_lex(dims, c, mu, 3)
        gd = lambda idx: np.conj(np.swapaxes(g[idx], 1, 2))  # noqa: E731
        assert np.abs(fat2[:, mu] - g @ fat[:, mu] @ gd(n1)).max() < 1e-13
        assert np.abs(lng2[:, mu] - g @ lng[:, mu] @ gd(n3)).max() < 1e-13


def test_rng_is_counter_based():
    """A sub-range of the variates equals the same slice of the full stream."""
    full = synth.counter_normals(7, 3, 1000)
    from synth.gauge import counter_normals_range

    assert np.array_equal(full[400:700], counter_normals_range(7, 3, 400, 300))
    assert abs(full.mean()) < 0.15 and abs(full.std() - 1.0) < 0.1


# --------------------------------------------------------------- operator pins


@pytest.mark.parametrize("dims,momenta", [((4, 4, 4, 4), MOMENTA_4), ((4, 6, 8, 10), MOMENTA_ASYM)])
@pytest.mark.parametrize("c1,c3", [(C1_ASQTAD, C3_ASQTAD), (1.0, 0.0), (0.0, 1.0)])
def test_free_field_closed_form(dims, momenta, c1, c3):
    """Unit-matrix links F = c1, L = c3: M e^{ipx} = (m^2 + sum (c1 sin p + c3 sin 3p)^2) e^{ipx}."""
    assert free_field_error(dims, c1, c3, 0.1, momenta) < 1e-13


def test_free_field_through_link_recipe():
    """The eps = 0 links of the workload recipe are the free field with (7/4, -1/24)."""
    dims = (4, 6, 8, 10)
    fat, lng = synth.gauge_field(dims, 0.0, 5)
    assert free_field_error(dims, 1.75, -1.0 / 24.0, 0.05, MOMENTA_ASYM, fat, lng) < 1e-13


def test_free_field_dense_spectrum_4444():
    """Whole spectrum of the dense 384x384 free M on 4^4 equals the closed-form multiset."""
    dims = (4, 4, 4, 4)
    mass = 0.2
    fat, lng = _unit_links(dims, C1_ASQTAD, C3_ASQTAD)
    n = (int(np.prod(dims)) // 2) * 3
    M = oracle.dense_matrix(lambda v: oracle.apply_m(fat, lng, v.reshape(-1, 3), mass, dims).ravel(), n)
    ev = np.sort(np.linalg.eigvalsh(M))
    lam = []
    for idx in np.ndindex(*dims):
        p = 2 * np.pi * np.asarray(idx) / np.asarray(dims)
        lam.append(mass * mass + _free_eigenvalue(p, C1_ASQTAD, C3_ASQTAD))
    lam = np.sort(lam)[::2]  # p and p + (pi,pi,pi,pi) coincide on even sites
    expect = np.sort(np.repeat(lam, 3))
    assert np.abs(ev - expect).max() < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 4, 8)])
def test_antihermiticity(dims):
    fat, lng = synth.gauge_field(dims, 0.3, 1003)
    assert antihermiticity_error(dims, fat, lng) < 1e-14


@pytest.mark.parametrize("out_parity", [0, 1])
def test_gauge_covariance(out_parity):
    assert covariance_error((4, 4, 6, 4), 0.3, 1004, out_parity) < 1e-13


def test_normal_operator_is_hpd():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, 1005)
    n = 128 * 3
    M = oracle.dense_matrix(lambda v: oracle.apply_m(fat, lng, v.reshape(-1, 3), 0.1, dims).ravel(), n)
    assert np.abs(M - M.conj().T).max() < 1e-13
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= 0.01 - 1e-12


def test_sampled_sites_match_full_apply():
    dims = (4, 6, 4, 8)
    fat, lng = synth.gauge_field(dims, 0.3, 1006)
    psi = synth.random_spinor(dims, 4)
    full = oracle.dslash(fat, lng, psi, dims, 1)
    sites = np.array([0, 5, 17, 95, 191])
    assert np.array_equal(oracle.dslash(fat, lng, psi, dims, 1, out_sites=sites), full[sites])


def test_apply_m_at_sites_matches_full_apply():
    dims = (4, 6, 4, 8)
    fat, lng = synth.gauge_field(dims, 0.3, 1008)
    v = synth.random_spinor(dims, 12)
    full = oracle.apply_m(fat, lng, v, 0.07, dims, shift=0.03)
    sites = np.array([0, 3, 50, 191])
    part = oracle.apply_m_at_sites(fat, lng, v, 0.07, dims, sites, shift=0.03)
    assert np.abs(part - full[sites]).max() < 1e-14


# --------------------------------------------------------------- solver pins


@pytest.fixture(scope="module")
def dense_4444():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, 1007)
    mass = 0.1
    n = 128 * 3
    M = oracle.dense_matrix(lambda v: oracle.apply_m(fat, lng, v.reshape(-1, 3), mass, dims).ravel(), n)
    b = synth.gaussian_source(dims, 5000)
    return dims, fat, lng, mass, M, b


def test_cg_matches_dense_solve(dense_4444):
    dims, fat, lng, mass, M, b = dense_4444
    x, info = oracle.cg(fat, lng, b, mass, dims, tol=1e-10)
    xd = np.linalg.solve(M, b.ravel())
    assert info["converged"] and info["true_rel_resid"] <= 1e-10
    # independent residual through the dense matrix
    assert np.linalg.norm(M @ x.ravel() - b.ravel()) / np.linalg.norm(b) <= 1e-10
    assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-8


def test_cg_initial_guess_and_shift(dense_4444):
    dims, fat, lng, mass, M, b = dense_4444
    shift = 0.05
    xd = np.linalg.solve(M + shift * np.eye(M.shape[0]), b.ravel())
    x0 = (xd + 1e-3 * synth.random_spinor(dims, 9).ravel()).reshape(-1, 3)
    x, info = oracle.cg(fat, lng, b, mass, dims, tol=1e-12, x0=x0, shift=shift)
    assert info["converged"]
    assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-10


def test_multishift_matches_dense_solves(dense_4444):
    dims, fat, lng, mass, M, b = dense_4444
    shifts = [10 ** (-4 + k / 2) for k in range(9)]
    xs, infos = oracle.multishift_cg(fat, lng, b, mass, shifts, dims, tol=1e-10)
    n = M.shape[0]
    for s, x, inf in zip(shifts, xs, infos):
        xd = np.linalg.solve(M + s * np.eye(n), b.ravel())
        assert inf["converged"] and inf["refine_iters"] == 0
        assert np.linalg.norm((M + s * np.eye(n)) @ x.ravel() - b.ravel()) / np.linalg.norm(b) <= 1e-10
        assert np.linalg.norm(x.ravel() - xd) / np.linalg.norm(xd) < 1e-8
    # larger shifts are better conditioned and stop earlier
    its = [inf["iters"] for inf in infos]
    assert its == sorted(its, reverse=True)


def test_multishift_unsorted_shifts_match_cg(dense_4444):
    dims, fat, lng, mass, M, b = dense_4444
    shifts = [0.3, 0.0, 0.02]
    xs, infos = oracle.multishift_cg(fat, lng, b, mass, shifts, dims, tol=1e-11)
    for s, x in zip(shifts, xs):
        xc, _ = oracle.cg(fat, lng, b, mass, dims, tol=1e-11, shift=s)
        assert np.linalg.norm(x - xc) / np.linalg.norm(xc) < 1e-8


# --------------------------------------------------------------- planted slips


def _wrong_phase(mu, c):
    # eta depending on the coordinate along mu itself
    return np.where(c[:, mu] % 2 == 0, 1.0, -1.0)


def _no_dagger(m):
    return m


def test_planted_wrong_phase_fails_free_field(monkeypatch):
    monkeypatch.setattr(ost, "staggered_phase", _wrong_phase)
    assert free_field_error((4, 6, 8, 10), C1_ASQTAD, C3_ASQTAD, 0.1, MOMENTA_ASYM) > 1e-3


def test_planted_missing_dagger_fails_antihermiticity(monkeypatch):
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, 1003)
    monkeypatch.setattr(ost, "_dag", _no_dagger)
    assert antihermiticity_error(dims, fat, lng) > 1e-3


def test_planted_wrong_backward_site_fails_covariance(monkeypatch):
    """Backward Naik hop taking L(x)^dag instead of L(x-3mu)^dag."""
    real = ost.neighbour_lex

    def patched(fat, lng, psi, dims, out_parity, out_sites=None):
        dims = tuple(dims)
        lex_out = ost.parity_sites(dims, out_parity)
        c = ost.site_coords(dims, lex_out)
        out = np.zeros((len(lex_out), 3), dtype=np.complex128)
        for mu in range(4):
            eta = ost.staggered_phase(mu, c)
            for links, hop in ((fat, 1), (lng, 3)):
                fwd = real(dims, c, mu, +hop)
                bwd = real(dims, c, mu, -hop)
                lb = lex_out if hop == 3 else bwd
                f = np.einsum("nij,nj->ni", links[lex_out, mu], psi[fwd // 2])
                b = np.einsum("nij,nj->ni", ost._dag(links[lb, mu]), psi[bwd // 2])
                out += eta[:, None] * (f - b)
        return 0.5 * out

    monkeypatch.setattr(ost, "dslash", patched)
    monkeypatch.setattr(oracle, "dslash", patched)
    assert covariance_error((4, 4, 6, 4), 0.3, 1004, 0) > 1e-3


def test_planted_dropped_naik_backward_fails_free_field(monkeypatch):
    real_einsum = np.einsum
    calls = {"n": 0}

    def patched(fat, lng, psi, dims, out_parity, out_sites=None):
        dims = tuple(dims)
        lex_out = ost.parity_sites(dims, out_parity)
        c = ost.site_coords(dims, lex_out)
        out = np.zeros((len(lex_out), 3), dtype=np.complex128)
        for mu in range(4):
            eta = ost.staggered_phase(mu, c)
            for links, hop in ((fat, 1), (lng, 3)):
                fwd = ost.neighbour_lex(dims, c, mu, +hop)
                bwd = ost.neighbour_lex(dims, c, mu, -hop)
                f = real_einsum("nij,nj->ni", links[lex_out, mu], psi[fwd // 2])
                b = real_einsum("nij,nj->ni", ost._dag(links[bwd, mu]), psi[bwd // 2])
                out += eta[:, None] * (f - (0 if hop == 3 else b))
        calls["n"] += 1
        return 0.5 * out

    monkeypatch.setattr(ost, "dslash", patched)
    assert free_field_error((4, 6, 8, 10), C1_ASQTAD, C3_ASQTAD, 0.1, MOMENTA_ASYM) > 1e-3
    assert calls["n"] > 0


# ------------------------------------------------- Lanczos estimate of kappa


def _cg_coefficients(A, b, steps):
    """alpha_j and beta_j of plain CG on a small dense SPD matrix (test-side)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    al, be = [], []
    for _ in range(steps):
        Ap = A @ p
        a = rr / (p @ Ap)
        x += a * p
        r -= a * Ap
        rr_new = r @ r
        al.append(a)
        be.append(rr_new / rr)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return al, be


def test_lanczos_ritz_values_recover_a_diagonal_spectrum():
    """n CG steps on an n x n matrix with distinct eigenvalues: the Lanczos
    tridiagonal is similar to the matrix, so its eigenvalues are exactly the
    matrix's (Golub and Van Loan, Sec. 10.2)."""
    d = np.array([0.5, 1.0, 2.5, 4.0, 7.0, 11.0])
    al, be = _cg_coefficients(np.diag(d), np.ones(6), 6)
    np.testing.assert_allclose(oracle.staggered.lanczos_ritz_values(al, be), d, rtol=1e-10)


def test_cg_ritz_values_bracket_the_dense_spectrum(dense_4444):
    """The oracle CG's Ritz values lie inside [lambda_min, lambda_max] of the
    dense 4^4 operator, and the extremes converge to them: kappa_est is the
    condition number that numpy.linalg.eigvalsh gives."""
    dims, fat, lng, mass, M, b = dense_4444
    lam = np.linalg.eigvalsh(M)
    _, info = oracle.cg(fat, lng, b, mass, dims, tol=1e-12)
    r = info["ritz"]
    assert lam[0] * (1 - 1e-12) <= r[0] and r[-1] <= lam[-1] * (1 + 1e-12)
    assert abs(r[-1] - lam[-1]) < 1e-12 * lam[-1]
    assert abs(r[0] - lam[0]) < 1e-6 * lam[0]
    assert abs(info["kappa_est"] - lam[-1] / lam[0]) < 1e-6 * lam[-1] / lam[0]


def test_planted_lanczos_error_fails_closed_form(monkeypatch):
    def broken(alphas, betas):  # off-diagonal without the square root
        k = len(alphas)
        T = np.zeros((k, k))
        for j in range(k):
            T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
            if j + 1 < k:
                T[j, j + 1] = T[j + 1, j] = betas[j] / alphas[j]
        return np.linalg.eigvalsh(T)

    monkeypatch.setattr(oracle.staggered, "lanczos_ritz_values", broken)
    with pytest.raises(AssertionError):
        test_lanczos_ritz_values_recover_a_diagonal_spectrum()
