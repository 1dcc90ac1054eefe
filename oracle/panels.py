"""Flat-triangle panel geometry (oracle; test infrastructure only).

Constant panels with collocation at the centroid ("center of every panel",
Sec. 3.2); S_j is the triangle area and the unit normal is the right-hand
normal (b - a) x (c - a) / |...| (outward for the counter-clockwise meshes of
synth/). Pinned by: the areas of the refined icosahedron summing to less than
and converging to 4 pi, normals pointing along the centroid on a sphere
(tests/test_oracle_bem.py).
"""
import numpy as np


def panel_vertices(vertices, triangles):
    """[n, 9] array of each panel's three vertices (the layout the C oracle reads)."""
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles)
    return np.ascontiguousarray(v[t].reshape(len(t), 9))


def geometry(vertices, triangles):
    v = np.asarray(vertices, dtype=np.float64)
    t = np.asarray(triangles)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    cr = np.cross(b - a, c - a)
    ln = np.linalg.norm(cr, axis=1)
    return (a + b + c) / 3.0, cr / ln[:, None], 0.5 * ln

