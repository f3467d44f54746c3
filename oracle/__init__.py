"""FP64 CPU oracle for the improved-staggered even-odd solve (test infrastructure).

This package is test infrastructure.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and the
library shares no code with it (no kernels, helpers, tables or constants).
It is plain numpy in float64/complex128, written for a reader to check
against the definitions by eye, not for speed.

Parity status of each function (what pins it, checked by the CPU tests):
  * dslash / apply_m       -- free-field closed form on plane waves,
                              anti-hermiticity D_eo = -D_oe^dag, gauge
                              covariance under random SU(3) transforms, full
                              free-field spectrum of a dense 4^4 build.
  * cg                     -- dense LU solve (numpy.linalg.solve) on 4^4;
                              its Lanczos Ritz values / kappa estimate
                              (lanczos_ritz_values) by the exact spectrum of
                              a diagonal matrix after n steps and by the
                              dense 4^4 spectrum (numpy.linalg.eigvalsh).
  * multishift_cg          -- dense LU solve per shift on 4^4, and single-mass
                              CG run shift by shift.
  * true_residual          -- exact definition ||b - M x|| / ||b||.
  * network (module)       -- forward, backward and loss of the gauge-covariant
                              preconditioner network: finite differences of
                              the loss, transport adjointness, gauge
                              covariance (tests/test_network_oracle.py).
  * apply_m_at_sites       -- equals apply_m restricted to the sampled sites
                              (checked on small lattices), used to check
                              full-size GPU results site by site.
  * links (module)         -- fat and Naik links from thin links: unit-link
                              closed form, single-link insertion at the sites
                              the definition names, gauge covariance
                              (tests/test_links_oracle.py).
  * gauge_force (module)   -- Symanzik one-loop gauge force: finite
                              differences of the action per loop type, unit
                              links, gauge covariance
                              (tests/test_gauge_force_oracle.py).
  * fermion_force (module) -- fermion force of a multi-shift pseudofermion
                              action through the fat and Naik links: finite
                              differences of the action (solved with cg) per
                              term type, gauge covariance, planted errors
                              caught (tests/test_fermion_force_oracle.py).
"""

from .staggered import (
    staggered_phase,
    site_coords,
    parity_sites,
    neighbour_lex,
    dslash,
    apply_m,
    apply_m_at_sites,
    true_residual,
    cg,
    multishift_cg,
    dense_matrix,
)

__all__ = [
    "staggered_phase",
    "site_coords",
    "parity_sites",
    "neighbour_lex",
    "dslash",
    "apply_m",
    "apply_m_at_sites",
    "true_residual",
    "cg",
    "multishift_cg",
    "dense_matrix",
]
