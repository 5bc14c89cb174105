"""Seeded synthetic inputs: structured tetrahedral cube meshes, coefficient fields and
node partitions.

This package only builds inputs (geometry, connectivity, coefficients, owner labels).
It holds none of the reduced-basis method's arithmetic: no element matrices, no
subdomain extension, no solves.  Both the CUDA path and the CPU oracle consume the
arrays produced here.
"""
from .meshes import (  # noqa: F401
    Mesh,
    kuhn_cube,
    lognormal_kappa,
    sphere_kappa,
    sine_kappa,
    box_owner,
    slab_owner,
    kmeans_owner,
    kuhn_box_tets,
    box_node_range,
    workload,
    WORKLOADS,
)
