"""FP64 oracle of the staggered fermion force through the link construction
(test infrastructure).

The paper benchmarks the HISQ fermion force of the RHMC/RHMD algorithm as its
third routine (Sec. 4.2, last part) without printing it.  The oracle writes
out the derivative it stands for, for the smearing used here (three-staple
fat link and Naik link built from the thin links, as in oracle/links.py):

    S(U) = sum_i alpha_i  phi^dag (M + sigma_i)^{-1} phi,
    M = m^2 - D_eo D_oe   (even sites),

the pseudofermion action of a rational approximation in partial fractions.
With X_i = (M + sigma_i)^{-1} phi (even sites) and Y_i = D_oe X_i (odd sites),
and D anti-Hermitian, a change of the links changes S by

    dS = sum_i alpha_i 2 Re( X_i^dag dD_eo Y_i ).

Writing out D (1/2, staggered phases eta, hops 1 and 3) turns this into a sum
over fat and Naik links:

    dS = sum_{x, mu} Re Tr[ dF_mu(x) G^F_mu(x) ] + Re Tr[ dL_mu(x) G^L_mu(x) ]

with the outer-product fields, summed over i with weight alpha_i,

    x even:  G^F_mu(x) =  eta_mu(x) Y(x+mu) X(x)^dag,   G^L_mu(x) =  eta_mu(x) Y(x+3mu) X(x)^dag
    x odd:   G^F_mu(x) = -eta_mu(x) X(x+mu) Y(x)^dag,   G^L_mu(x) = -eta_mu(x) X(x+3mu) Y(x)^dag

(eta_mu is unchanged along mu, so the backward hops give the odd-site terms).
The chain rule through the link construction then collects, for every thin
link, Z_nu(y) with dS = sum Re Tr[ dU_nu(y) Z_nu(y) ]: a product
A_1 ... A_n of thin links (each forward, or daggered) weighted by G gives,
for its factor k with left part P = A_1..A_{k-1} and right part Q =
A_{k+1}..A_n, Re Tr[P dA_k Q G] = Re Tr[dA_k (Q G P)], so

    A_k = U        ->  Z += Q G P
    A_k = U^dag    ->  Z += (Q G P)^dag.

Moving one link as U -> exp(eps X) U (X traceless anti-Hermitian), dU = X U
and dS/deps = Re Tr[X U Z] = -Re Tr[X F] with

    F_nu(y) = -TA[ U_nu(y) Z_nu(y) ],  TA(A) = (A - A^dag)/2 - Tr(A - A^dag)/6,

the sign convention of the gauge-force oracle.

The factor lists of the fat and Naik links are written out once below
(``link_terms``) and reused both to build the links (checked against
oracle/links.py) and to differentiate them.

Parity status (tests/test_fermion_force_oracle.py): link_terms rebuild
exactly the fat and Naik links of oracle/links.py; finite differences of the
action S (two shifts, every link product on) along random X on single links
of a 6^4 lattice match -Re Tr(X F), separately for the one-link, staple and
Naik terms; gauge covariance F_nu(y) -> G(y) F_nu(y) G(y)^dag; a planted
error (one staple factor's dagger dropped, or a sign of G flipped) fails the
finite-difference pin.
"""

import numpy as np

from .links import fat_links, naik_links
from .staggered import cg, dslash, neighbour_lex, site_coords, staggered_phase


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def traceless_antihermitian(A):
    B = 0.5 * (A - _dag(A))
    return B - (np.trace(B, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)


def link_terms(dims, c1, c_st, c3):
    """The fat and Naik links as sums of products of thin links.

    Returns {"fat": {mu: [...]}, "naik": {mu: [...]}}; every entry is
    (coefficient, [(lex site array, direction, dagger), ...]): the factors of
    one product for all output sites x (lex order), left to right.
    """
    V = int(np.prod(dims))
    x = np.arange(V)
    c = site_coords(dims, x)
    out = {"fat": {}, "naik": {}}
    for mu in range(4):
        x_pmu = neighbour_lex(dims, c, mu, +1)
        x_p2mu = neighbour_lex(dims, c, mu, +2)
        terms = [(c1, [(x, mu, False)])]
        for nu in range(4):
            if nu == mu:
                continue
            x_pnu = neighbour_lex(dims, c, nu, +1)
            x_mnu = neighbour_lex(dims, c, nu, -1)
            x_mnu_pmu = neighbour_lex(dims, site_coords(dims, x_mnu), mu, +1)
            # upper staple U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
            terms.append((c_st, [(x, nu, False), (x_pnu, mu, False), (x_pmu, nu, True)]))
            # lower staple U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
            terms.append((c_st, [(x_mnu, nu, True), (x_mnu, mu, False), (x_mnu_pmu, nu, False)]))
        out["fat"][mu] = terms
        out["naik"][mu] = [(c3, [(x, mu, False), (x_pmu, mu, False), (x_p2mu, mu, False)])]
    return out


def _factor(U, site, d, dag):
    m = U[site, d]
    return _dag(m) if dag else m


def build_from_terms(U, terms):
    """Evaluate a term list of link_terms into [V][4][3][3]."""
    V = U.shape[0]
    out = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    for mu, tl in terms.items():
        for coef, factors in tl:
            P = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 3, 3))
            for site, d, dag in factors:
                P = P @ _factor(U, site, d, dag)
            out[:, mu] += coef * P
    return out


def outer_products(xs, ys, alphas, dims):
    """G^F and G^L ([V][4][3][3]) from even fields xs[i] and odd fields ys[i]
    ([V/2][3], checkerboard index lex // 2), weights alphas[i]."""
    V = int(np.prod(dims))
    lex = np.arange(V)
    c = site_coords(dims, lex)
    even = c.sum(axis=1) % 2 == 0
    GF = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    GL = np.zeros_like(GF)
    for X, Y, a in zip(xs, ys, alphas):
        for mu in range(4):
            eta = staggered_phase(mu, c)
            for G, hop in ((GF, 1), (GL, 3)):
                nb = neighbour_lex(dims, c, mu, hop)
                # even x: Y(x+hop) X(x)^dag; odd x: -X(x+hop) Y(x)^dag
                left = np.where(even[:, None], Y[nb // 2], X[nb // 2])
                right = np.where(even[:, None], X[lex // 2], Y[lex // 2])
                sign = np.where(even, 1.0, -1.0) * eta
                G[:, mu] += (a * sign)[:, None, None] * np.einsum("ni,nj->nij", left, np.conj(right))
    return GF, GL


def link_gradient(U, GF, GL, dims, c1, c_st, c3):
    """Z with dS = sum Re Tr[dU_nu(y) Z_nu(y)] for dS = sum Re Tr[dF G^F + dL G^L]."""
    V = U.shape[0]
    Z = np.zeros_like(U)
    terms = link_terms(dims, c1, c_st, c3)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 3, 3))
    for kind, G in (("fat", GF), ("naik", GL)):
        for mu, tl in terms[kind].items():
            for coef, factors in tl:
                mats = [_factor(U, s, d, dag) for s, d, dag in factors]
                for k, (site, d, dag) in enumerate(factors):
                    P = eye
                    for m in mats[:k]:
                        P = P @ m
                    Q = eye
                    for m in mats[k + 1 :]:
                        Q = Q @ m
                    C = coef * (Q @ G[:, mu] @ P)
                    np.add.at(Z[:, d], site, _dag(C) if dag else C)
    return Z


def fermion_force(U, xs, ys, alphas, dims, c1=1.0, c_st=0.125, c3=-1.0 / 24.0):
    """F_nu(y) = -TA[U_nu(y) Z_nu(y)], [V][4][3][3], for solution pairs
    (X_i even, Y_i = D_oe X_i odd) with weights alpha_i."""
    GF, GL = outer_products(xs, ys, alphas, dims)
    Z = link_gradient(U, GF, GL, dims, c1, c_st, c3)
    return -traceless_antihermitian(U @ Z)


def solutions(U, phi, mass, shifts, dims, c1=1.0, c_st=0.125, c3=-1.0 / 24.0, tol=1e-13):
    """X_i = (M + sigma_i)^{-1} phi and Y_i = D_oe X_i on the links built from U."""
    fat = fat_links(U, dims, c1, c_st)
    lng = naik_links(U, dims, c3)
    xs, ys = [], []
    for s in shifts:
        X, info = cg(fat, lng, phi, mass, dims, tol=tol, shift=s)
        assert info["converged"], info
        xs.append(X)
        ys.append(dslash(fat, lng, X, dims, out_parity=1))
    return xs, ys


def action(U, phi, mass, shifts, alphas, dims, c1=1.0, c_st=0.125, c3=-1.0 / 24.0, tol=1e-13):
    """S = sum_i alpha_i Re phi^dag (M + sigma_i)^{-1} phi on the links built from U."""
    xs, _ = solutions(U, phi, mass, shifts, dims, c1, c_st, c3, tol)
    return float(sum(a * np.vdot(phi.ravel(), X.ravel()).real for a, X in zip(alphas, xs)))
