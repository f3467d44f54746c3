"""FP64 oracle of the even-odd improved-staggered operator and its CG solvers.

Test infrastructure only (see the package docstring): plain numpy, complex128.

The paper benchmarks the staggered single-mass and multi-shift conjugate
gradient (Sec. 1, Sec. 4 and Sec. 4.1: "the most time-consuming part of the
code in production runs"; arithmetic intensity 0.26 flop/byte, Sec. 4.2) but
does not print the operator.  The oracle writes out the standard
improved-staggered (asqtad-form) operator it refers to:

    (D psi)(x) = 1/2 sum_mu eta_mu(x) [ F_mu(x) psi(x+mu) - F_mu(x-mu)^dag psi(x-mu)
                                       + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^dag psi(x-3mu) ]

with fat links F, Naik links L, staggered phases eta_x = 1,
eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z), periodic wrap in
all four directions.  D couples only opposite parities (both hop lengths are
odd), D_oe maps even-site fields to odd sites and D_eo the reverse, and the
even-site normal operator is

    M = m^2 - D_eo D_oe          (Hermitian positive definite, D_eo = -D_oe^dag).

Conventions of the canonical layout are those of :mod:`synth.gauge`: lex
order with x fastest, single-parity fields indexed by lex // 2.
"""

import numpy as np


# ----------------------------------------------------------------- indexing


def site_coords(dims, lex):
    """(n, 4) integer coordinates (x, y, z, t) of lexicographic site indices."""
    Lx, Ly, Lz, Lt = dims
    lex = np.asarray(lex, dtype=np.int64)
    x = lex % Lx
    y = (lex // Lx) % Ly
    z = (lex // (Lx * Ly)) % Lz
    t = lex // (Lx * Ly * Lz)
    return np.stack([x, y, z, t], axis=1)


def lex_of(dims, c):
    """Lexicographic index of (n, 4) coordinates."""
    Lx, Ly, Lz, _ = dims
    return c[:, 0] + Lx * (c[:, 1] + Ly * (c[:, 2] + Lz * c[:, 3]))


def parity_sites(dims, parity):
    """Lex indices of all sites with (x+y+z+t) % 2 == parity, in checkerboard order.

    The checkerboard index of such a site is lex // 2; listing the sites in
    increasing lex order lists them in increasing checkerboard index.
    """
    V = int(np.prod(dims))
    lex = np.arange(V, dtype=np.int64)
    par = site_coords(dims, lex).sum(axis=1) % 2
    return lex[par == parity]


def neighbour_lex(dims, c, mu, k):
    """Lex index of the site c + k * mu_hat with periodic wrap."""
    n = c.copy()
    n[:, mu] = (n[:, mu] + k) % dims[mu]
    return lex_of(dims, n)


def staggered_phase(mu, c):
    """eta_mu(x): 1, (-1)^x, (-1)^(x+y), (-1)^(x+y+z) for mu = x, y, z, t."""
    s = c[:, :mu].sum(axis=1) if mu > 0 else np.zeros(len(c), dtype=np.int64)
    return np.where(s % 2 == 0, 1.0, -1.0)


# ----------------------------------------------------------------- operator


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def dslash(fat, lng, psi, dims, out_parity, out_sites=None):
    """(D psi)(x) on the sites x of parity ``out_parity``.

    fat, lng : [V][4][3][3] complex128 links (no phases folded in).
    psi      : [V/2][3] complex128 field on the opposite parity.
    out_sites: optional checkerboard indices of the output sites to compute
               (all of them if None); the result has one row per entry.
    """
    dims = tuple(dims)
    lex_out = parity_sites(dims, out_parity)
    if out_sites is not None:
        lex_out = lex_out[np.asarray(out_sites, dtype=np.int64)]
    c = site_coords(dims, lex_out)
    out = np.zeros((len(lex_out), 3), dtype=np.complex128)
    for mu in range(4):
        eta = staggered_phase(mu, c)
        for links, hop in ((fat, 1), (lng, 3)):
            fwd = neighbour_lex(dims, c, mu, +hop)
            bwd = neighbour_lex(dims, c, mu, -hop)
            forward = np.einsum("nij,nj->ni", links[lex_out, mu], psi[fwd // 2])
            backward = np.einsum("nij,nj->ni", _dag(links[bwd, mu]), psi[bwd // 2])
            out += eta[:, None] * (forward - backward)
    return 0.5 * out


def apply_m(fat, lng, v, mass, dims, shift=0.0):
    """(m^2 + shift) v - D_eo D_oe v for an even-site field v ([V/2][3])."""
    t = dslash(fat, lng, v, dims, out_parity=1)
    return (mass * mass + shift) * v - dslash(fat, lng, t, dims, out_parity=0)


def apply_m_at_sites(fat, lng, v, mass, dims, sites, shift=0.0):
    """((m^2 + shift) v - D_eo D_oe v) at the even checkerboard sites `sites` only.

    D_oe v is evaluated only on the odd neighbours (distance 1 and 3 in every
    direction) of the requested sites, then D_eo on the requested sites: the
    same definition as :func:`apply_m`, restricted to what those outputs read.
    """
    dims = tuple(dims)
    sites = np.asarray(sites, dtype=np.int64)
    c = site_coords(dims, parity_sites(dims, 0)[sites])
    nb = [neighbour_lex(dims, c, mu, k) // 2 for mu in range(4) for k in (1, -1, 3, -3)]
    nb = np.unique(np.concatenate(nb))
    t = np.zeros_like(v)
    t[nb] = dslash(fat, lng, v, dims, out_parity=1, out_sites=nb)
    return (mass * mass + shift) * v[sites] - dslash(fat, lng, t, dims, out_parity=0, out_sites=sites)


def _dot(a, b):
    """<a, b> = sum conj(a) b."""
    return np.vdot(a.ravel(), b.ravel())


def true_residual(fat, lng, x, b, mass, dims, shift=0.0):
    """||b - (M + shift) x|| / ||b|| in FP64."""
    r = b - apply_m(fat, lng, x, mass, dims, shift)
    return float(np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel()))


# ----------------------------------------------------------------- solvers


def cg(fat, lng, b, mass, dims, tol=1e-10, max_iter=100000, x0=None, shift=0.0):
    """Conjugate gradient (Hestenes-Stiefel) on (M + shift) x = b in FP64.

    Iterates until the recursively updated residual satisfies
    ||r|| <= tol ||b||, then recomputes r = b - A x; if that true residual
    still exceeds the target, CG continues from (x, r_true).
    Returns (x, info) with info = {iters, true_rel_resid, converged,
    ritz, kappa_est}: the eigenvalues of the Lanczos tridiagonal that CG's
    alpha and beta define (up to the first true-residual restart, after
    which the recurrence is no longer a Lanczos one), and the ratio of the
    largest to the smallest, an estimate of the condition number of
    (M + shift) from below.
    """
    A = lambda v: apply_m(fat, lng, v, mass, dims, shift)  # noqa: E731
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128, copy=True)
    r = b - A(x) if x0 is not None else b.copy()
    p = r.copy()
    bb = _dot(b, b).real
    rr = _dot(r, r).real
    target = tol * tol * bb
    it = 0
    converged = rr <= target
    alphas, betas, lanczos = [], [], True
    while not converged and it < max_iter:
        Ap = A(p)
        pAp = _dot(p, Ap).real
        alpha = rr / pAp
        x += alpha * p
        r -= alpha * Ap
        rr_new = _dot(r, r).real
        it += 1
        if lanczos:
            alphas.append(alpha)
        if rr_new <= target:
            r = b - A(x)
            rr_new = _dot(r, r).real
            converged = rr_new <= target
            lanczos = False
        beta = rr_new / rr
        if lanczos:
            betas.append(beta)
        p = r + beta * p
        rr = rr_new
    res = true_residual(fat, lng, x, b, mass, dims, shift)
    ritz = lanczos_ritz_values(alphas, betas)
    info = {"iters": it, "true_rel_resid": res, "converged": res <= tol, "ritz": ritz,
            "kappa_est": float(ritz[-1] / ritz[0]) if len(ritz) else float("nan")}
    return x, info


def lanczos_ritz_values(alphas, betas):
    """Eigenvalues (ascending) of the Lanczos tridiagonal T_k of k CG steps.

    CG's coefficients define it (Golub and Van Loan, Sec. 10.2; Saad,
    Iterative Methods, Sec. 6.7.3): with alpha_j the step lengths and
    beta_j = |r_{j+1}|^2 / |r_j|^2,
        T_jj     = 1/alpha_j + beta_{j-1}/alpha_{j-1}   (second term absent for j = 0)
        T_j,j+1  = sqrt(beta_j) / alpha_j.
    Only the betas of steps followed by another step enter the off-diagonal.
    """
    k = len(alphas)
    if k == 0:
        return np.zeros(0)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return np.linalg.eigvalsh(T)


def multishift_cg(fat, lng, b, mass, shifts, dims, tol=1e-10, max_iter=100000):
    """Multi-shift CG for (M + sigma_s) x_s = b, all shifts from one Krylov space.

    The base system is the smallest shift sigma_0.  With Delta_s = sigma_s -
    sigma_0 the shifted residuals stay collinear with the base one,
    r_s = zeta_s r, and the scalars follow from matching the three-term
    residual recurrence of CG (Jegerlehner's shifted-CG relations):

        zeta_s(k+1) = zeta_s(k) zeta_s(k-1) a(k-1) /
                      [ a(k-1) zeta_s(k-1) (1 + a(k) Delta_s)
                        + a(k) b(k-1) (zeta_s(k-1) - zeta_s(k)) ]
        a_s(k) = a(k) zeta_s(k+1) / zeta_s(k)
        b_s(k) = b(k) (zeta_s(k+1) / zeta_s(k))^2
        x_s += a_s(k) p_s ;  p_s = zeta_s(k+1) r(k+1) + b_s(k) p_s

    with zeta(-1) = zeta(0) = 1, a(-1) = 1, b(-1) = 0.  Shift s stops when
    |zeta_s| ||r|| <= tol ||b||.  Every x_s is then checked with its FP64 true
    residual and, if it misses the target, refined by :func:`cg` from x_s.
    Returns (xs, info) with per-shift iteration counts and true residuals.
    """
    shifts = np.asarray(shifts, dtype=np.float64)
    order = np.argsort(shifts, kind="stable")
    s0 = shifts[order[0]]
    delta = shifts - s0
    ns = len(shifts)
    A0 = lambda v: apply_m(fat, lng, v, mass, dims, s0)  # noqa: E731
    bb = _dot(b, b).real
    r = b.copy()
    rr = bb
    xs = [np.zeros_like(b) for _ in range(ns)]
    ps = [b.copy() for _ in range(ns)]
    zeta_prev = np.ones(ns)
    zeta = np.ones(ns)
    alpha_prev, beta_prev = 1.0, 0.0
    active = np.ones(ns, dtype=bool)
    iters = np.zeros(ns, dtype=np.int64)
    it = 0
    while active.any() and it < max_iter:
        p = ps[order[0]]
        Ap = A0(p)
        alpha = rr / _dot(p, Ap).real
        zeta_next = zeta.copy()
        for s in range(ns):
            if not active[s]:
                continue
            den = alpha_prev * zeta_prev[s] * (1.0 + alpha * delta[s]) + alpha * beta_prev * (
                zeta_prev[s] - zeta[s]
            )
            zeta_next[s] = zeta[s] * zeta_prev[s] * alpha_prev / den
        r = r - alpha * Ap
        rr_new = _dot(r, r).real
        beta = rr_new / rr
        it += 1
        for s in range(ns):
            # the base direction drives the Krylov space and is always updated
            if not active[s] and s != order[0]:
                continue
            a_s = alpha * zeta_next[s] / zeta[s]
            b_s = beta * (zeta_next[s] / zeta[s]) ** 2
            if active[s]:
                xs[s] += a_s * ps[s]
                iters[s] = it
            ps[s] = zeta_next[s] * r + b_s * ps[s]
            if active[s] and abs(zeta_next[s]) * np.sqrt(rr_new) <= tol * np.sqrt(bb):
                active[s] = False
        zeta_prev, zeta = zeta, zeta_next
        alpha_prev, beta_prev = alpha, beta
        rr = rr_new
    infos = []
    for s in range(ns):
        res = true_residual(fat, lng, xs[s], b, mass, dims, shifts[s])
        refine = 0
        if res > tol:
            xs[s], inf = cg(fat, lng, b, mass, dims, tol, max_iter, x0=xs[s], shift=shifts[s])
            res, refine = inf["true_rel_resid"], inf["iters"]
        infos.append({"iters": int(iters[s]), "refine_iters": refine, "true_rel_resid": res, "converged": res <= tol})
    return xs, infos


# ----------------------------------------------------------------- dense forms


def dense_matrix(apply, n):
    """Dense matrix of a linear map on C^n by applying it to the unit vectors.

    ``apply`` takes and returns flat complex128 arrays of length n.
    """
    out = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        out[:, j] = apply(e)
        e[j] = 0.0
    return out
