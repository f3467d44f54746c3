"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package only *makes inputs*: random SU(3) gauge fields, the smeared
(fat) and three-link (Naik) fields built from them by the recipe the
benchmark workloads prescribe, and Gaussian colour-vector sources.  It holds
no arithmetic of the staggered Dirac operator (no staggered phases, no 1/2
normalisation, no hops) and none of the solvers.  Both sides receive the
same arrays from here.
"""

from .rng import counter_normals, counter_uniforms
from .gauge import (
    Lattice,
    random_su3,
    thin_links,
    fat_links,
    naik_links,
    gauge_field,
    gaussian_source,
    random_spinor,
    links_from_thin,
    random_gauge_transform,
    gauge_transform_links,
)

__all__ = [
    "counter_normals",
    "counter_uniforms",
    "Lattice",
    "random_su3",
    "thin_links",
    "fat_links",
    "naik_links",
    "gauge_field",
    "gaussian_source",
    "random_spinor",
    "links_from_thin",
    "random_gauge_transform",
    "gauge_transform_links",
]
