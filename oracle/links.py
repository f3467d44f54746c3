"""FP64 oracle of the link construction that precedes the staggered operator
(test infrastructure).

The paper's production code smears the thin gauge links before the solver
(HISQ-link smearing, Sec. 1; its share of the run time in Sec. 2, Fig. 1).
The workload here stands in a three-staple fat link and the Naik link:

    F_mu(x) = c1 U_mu(x)
              + c_st sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                                     + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
    L_mu(x) = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu)

with (c1, c_st, c3) = (1, 1/8, -1/24) in the benchmark workload.  Links are
canonical [V][4][3][3] complex128 in lex order (x fastest), periodic wrap.

Parity status (tests/test_links_oracle.py): unit links give the closed form
F = (c1 + 6 c_st) 1, L = c3 1; a single non-trivial link W enters exactly the
staples and Naik products that contain it, as W or W^dag, at the sites the
definition names; gauge covariance F_mu(x) -> G(x) F_mu(x) G(x+mu)^dag,
L_mu(x) -> G(x) L_mu(x) G(x+3mu)^dag under U_mu(x) -> G(x) U_mu(x) G(x+mu)^dag.
"""

import numpy as np

from .staggered import neighbour_lex, site_coords


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def fat_links(thin, dims, c1=1.0, c_st=0.125):
    """Three-staple fat links from thin links [V][4][3][3]."""
    V = thin.shape[0]
    c = site_coords(dims, np.arange(V))
    out = np.empty_like(thin)
    for mu in range(4):
        acc = c1 * thin[:, mu]
        x_pmu = neighbour_lex(dims, c, mu, +1)
        for nu in range(4):
            if nu == mu:
                continue
            x_pnu = neighbour_lex(dims, c, nu, +1)
            x_mnu = neighbour_lex(dims, c, nu, -1)
            x_mnu_pmu = neighbour_lex(dims, site_coords(dims, x_mnu), mu, +1)
            upper = thin[:, nu] @ thin[x_pnu, mu] @ _dag(thin[x_pmu, nu])
            lower = _dag(thin[x_mnu, nu]) @ thin[x_mnu, mu] @ thin[x_mnu_pmu, nu]
            acc = acc + c_st * (upper + lower)
        out[:, mu] = acc
    return out


def naik_links(thin, dims, c3=-1.0 / 24.0):
    """Naik links c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu) from thin links [V][4][3][3]."""
    V = thin.shape[0]
    c = site_coords(dims, np.arange(V))
    out = np.empty_like(thin)
    for mu in range(4):
        x1 = neighbour_lex(dims, c, mu, +1)
        x2 = neighbour_lex(dims, c, mu, +2)
        out[:, mu] = c3 * (thin[:, mu] @ thin[x1, mu] @ thin[x2, mu])
    return out
