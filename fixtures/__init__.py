"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds meshes, boundary masks, load descriptions and material
tables.  It holds none of the method's arithmetic (no shape functions, no
stresses, no assembly): only geometry, index bookkeeping and random draws.
"""
from .meshes import (  # noqa: F401
    Mesh,
    Material,
    kuhn_cube,
    artery_tube,
    mooney_rivlin,
    artery_layers,
    batched_tubes,
    batched_segment,
    cube_uniaxial_bc,
    tube_end_bc,
)
