"""Seeded synthetic inputs for the TL-FEA hot path.

This package builds meshes (structured hexahedral grids split into T4/T10
tetrahedra, or kept as H8 bricks), nodal displacement and velocity fields, and
material tables. It contains no finite-element arithmetic: no shape functions,
no quadrature, no stress. Both the CPU oracle (``oracle/``) and the CUDA path
consume what it produces, so it must stay free of the method itself.
"""

from .mesh import (  # noqa: F401
    T4, T10, H8, Q27, NODES_PER_ELEM, Mesh, box_mesh, concat_meshes, boundary_faces, face_corners,
)
from .workloads import (  # noqa: F401
    block_t10_svk, cantilever_beam, batch_bodies, diff_block, newton_beams,
    small_beam, lame_from_young, split_bodies, q27_beam,
)
