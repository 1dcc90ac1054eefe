"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package holds no arithmetic of the boundary-element method: it only builds
meshes (vertex coordinates and triangle connectivity) and seeded random vectors.
Panel centroids, normals, areas, quadrature points and all kernel evaluations are
computed separately by each side.
"""
from .mesh import (icosphere, octasphere, ellipsoid, evans_fung_cell, place_cells,
                   random_vector, point_charge_dirichlet, smooth_random_field)

__all__ = ["icosphere", "octasphere", "ellipsoid", "evans_fung_cell", "place_cells",
           "random_vector", "point_charge_dirichlet", "smooth_random_field"]
