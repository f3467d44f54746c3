"""FP64 oracle of the Symanzik one-loop improved gauge action and its force
(test infrastructure).

The paper benchmarks the "Symanzik one-loop gauge force" of the HISQ
RHMC/RHMD algorithm (Sec. 4.2, Figs. 6-8: matrix-matrix products, higher
arithmetic intensity than CG) without printing it.  The oracle writes out
the standard Luscher-Weisz form it refers to:

    S = beta sum_loops c_loop (1 - Re Tr W / 3)

over every plaquette (1x1, coefficient c_pl), every 1x2 rectangle (c_rt)
and every parallelogram -- the six-link loop a, b, c, -a, -b, -c around
three distinct directions (c_pg) -- each geometric loop counted once.

Force.  For the link U_mu(x), let Sigma_mu(x) = sum over loops W through
the link of c_loop times the product of W's other five (or three) links,
the loop oriented so that it starts with U_mu(x) traversed forward.  Moving
the link as U -> exp(eps X) U with X traceless anti-Hermitian changes the
action by dS/deps = -Re Tr(X F_mu(x)) with

    F_mu(x) = (beta / 3) TA[U_mu(x) Sigma_mu(x)],
    TA(M) = (M - M^dag)/2 - Tr(M - M^dag)/6.

Loop shapes are not written out by hand: every oriented closed path of a
family (a, b, -a, -b), (a, a, b, -a, -a, -b), (a, b, c, -a, -b, -c) over
signed distinct directions is reduced to its set of links relative to its
lowest corner, and duplicates are dropped; what remains, translated over
the lattice, is every geometric loop once.  The staples of a link are read
off the same shapes.

Parity status (tests/test_gauge_force_oracle.py): 6, 18 and 24 staples per
link; unit links give S = 0 and F = 0; finite differences of the action
along random X on single links match -Re Tr(X F); gauge covariance
F_mu(x) -> G(x) F_mu(x) G(x)^dag; a planted sign error fails the
finite-difference pin.
"""

import itertools

import numpy as np

from .staggered import lex_of, site_coords


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _steps_to_links(steps):
    """Links of a closed path of (direction, sign) steps from offset 0: a set of
    (base offset tuple, direction), the direction's link at that base."""
    pos = np.zeros(4, dtype=np.int64)
    links = []
    for d, s in steps:
        if s > 0:
            links.append((tuple(pos), d))
            pos[d] += 1
        else:
            pos[d] -= 1
            links.append((tuple(pos), d))
    assert not pos.any(), "path does not close"
    return links


def _canonical(links):
    base = np.min(np.array([o for o, _ in links]), axis=0)
    return frozenset((tuple(np.array(o) - base), d) for o, d in links)


def _families():
    signed = [(d, s) for d in range(4) for s in (1, -1)]
    neg = lambda st: (st[0], -st[1])  # noqa: E731
    fam = {"pl": [], "rt": [], "pg": []}
    for a, b in itertools.permutations(signed, 2):
        if a[0] == b[0]:
            continue
        fam["pl"].append([a, b, neg(a), neg(b)])
        fam["rt"].append([a, a, b, neg(a), neg(a), neg(b)])
    for a, b, c in itertools.permutations(signed, 3):
        if len({a[0], b[0], c[0]}) < 3:
            continue
        fam["pg"].append([a, b, c, neg(a), neg(b), neg(c)])
    return fam


def loop_shapes():
    """{kind: list of distinct loops, each a list of (direction, sign) steps from its start}."""
    out = {}
    for kind, paths in _families().items():
        seen = {}
        for p in paths:
            key = _canonical(_steps_to_links(p))
            seen.setdefault(key, p)
        out[kind] = list(seen.values())
    return out


def staple_paths():
    """{kind: {mu: list of (start offset of the staple, steps)}}: for each loop
    through U_mu(0), the path from 0 + mu back to 0 along the loop's other
    links, the loop oriented so that it traverses U_mu(0) forward."""
    out = {}
    for kind, loops in loop_shapes().items():
        out[kind] = {mu: [] for mu in range(4)}
        for steps in loops:
            n = len(steps)
            for orient in (steps, [(d, -s) for d, s in reversed(steps)]):
                # positions before each step
                pos = [np.zeros(4, dtype=np.int64)]
                for d, s in orient:
                    q = pos[-1].copy()
                    q[d] += s
                    pos.append(q)
                for i, (d, s) in enumerate(orient):
                    if s < 0:
                        continue
                    # rotate so the loop starts with this forward step; the staple
                    # is the rest, and the link sits at offset pos[i] of the loop
                    rest = orient[i + 1 :] + orient[:i]
                    out[kind][d].append((tuple(pos[i]), rest))
        # the same loop through the same link must appear once: translate every
        # staple so that its link is at the origin and drop duplicates
        for mu in range(4):
            uniq = {}
            for off, rest in out[kind][mu]:
                links = _steps_to_links([(mu, 1)] + rest)
                uniq.setdefault(frozenset(links), rest)
            out[kind][mu] = list(uniq.values())
    return out


def _path_product(U, dims, start, steps):
    """Product of the links along `steps` from the sites `start` (lex array)."""
    c = site_coords(dims, start)
    M = np.broadcast_to(np.eye(3, dtype=np.complex128), (len(start), 3, 3)).copy()
    for d, s in steps:
        if s > 0:
            M = M @ U[lex_of(dims, c), d]
            c = c.copy()
            c[:, d] = (c[:, d] + 1) % dims[d]
        else:
            c = c.copy()
            c[:, d] = (c[:, d] - 1) % dims[d]
            M = M @ _dag(U[lex_of(dims, c), d])
    return M


def action(U, dims, beta, c_pl, c_rt, c_pg):
    """S = beta sum over geometric loops c (1 - Re Tr W / 3)."""
    V = U.shape[0]
    sites = np.arange(V)
    coef = {"pl": c_pl, "rt": c_rt, "pg": c_pg}
    S = 0.0
    for kind, loops in loop_shapes().items():
        for steps in loops:
            W = _path_product(U, dims, sites, steps)
            S += beta * coef[kind] * np.sum(1.0 - np.real(np.trace(W, axis1=1, axis2=2)) / 3.0)
    return float(S)


def traceless_antihermitian(M):
    A = 0.5 * (M - _dag(M))
    tr = np.trace(A, axis1=-2, axis2=-1)
    return A - (tr / 3.0)[..., None, None] * np.eye(3)


def force(U, dims, beta, c_pl, c_rt, c_pg):
    """F_mu(x) = (beta/3) TA[U_mu(x) Sigma_mu(x)], [V][4][3][3]."""
    V = U.shape[0]
    sites = np.arange(V)
    c = site_coords(dims, sites)
    coef = {"pl": c_pl, "rt": c_rt, "pg": c_pg}
    F = np.empty_like(U)
    paths = staple_paths()
    for mu in range(4):
        cp = c.copy()
        cp[:, mu] = (cp[:, mu] + 1) % dims[mu]
        x_pmu = lex_of(dims, cp)
        Sig = np.zeros((V, 3, 3), dtype=np.complex128)
        for kind in ("pl", "rt", "pg"):
            for steps in paths[kind][mu]:
                Sig += coef[kind] * _path_product(U, dims, x_pmu, steps)
        F[:, mu] = (beta / 3.0) * traceless_antihermitian(U[:, mu] @ Sig)
    return F


def luscher_weisz_coefficients(u0):
    """Tadpole-improved one-loop coefficients (c_pl, c_rt, c_pg) for a mean
    link u0, with the coupling alpha_s = -4 ln(u0) / 3.0684 (the standard
    one-loop Symanzik values of the improved action)."""
    alpha_s = -4.0 * np.log(u0) / 3.0684
    return 1.0, -(1.0 + 0.4805 * alpha_s) / (20.0 * u0 * u0), -0.03325 * alpha_s / (u0 * u0)
