"""Triangulated surfaces and seeded vectors used as workloads.

Sphere meshes follow the paper's recipe (Sec. 3.1): start from a closed
polyhedron and split every triangle into four through its edge midpoints,
repeatedly. New vertices are projected onto the sphere. Triangles are
oriented counter-clockwise when seen from outside, so the right-hand normal
points out of the body.

Red-blood-cell surfaces apply the Evans-Fung biconcave map (Sec. 3.3, eq.
rbc_parameterization) to the vertices of a sphere mesh.
"""
import numpy as np

__all__ = ["icosphere", "octasphere", "ellipsoid", "evans_fung_cell", "place_cells",
           "random_vector", "point_charge_dirichlet"]


def _orient_outward(v, t):
    """Flip triangles whose right-hand normal points towards the origin."""
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    nrm = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    t = t.copy()
    t[flip, 1], t[flip, 2] = t[flip, 2].copy(), t[flip, 1].copy()
    return t


def _refine(v, t, levels, radius):
    """Split each triangle into four via edge midpoints, projecting onto the sphere."""
    v = [tuple(x) for x in v]
    t = [tuple(x) for x in t]
    for _ in range(levels):
        cache = {}

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            k = cache.get(key)
            if k is None:
                p = (np.asarray(v[i]) + np.asarray(v[j])) * 0.5
                p = p * (radius / np.linalg.norm(p))
                v.append(tuple(p))
                k = len(v) - 1
                cache[key] = k
            return k

        nt = []
        for (a, b, c) in t:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        t = nt
    return np.asarray(v, dtype=np.float64), np.asarray(t, dtype=np.int32)


def icosphere(levels, radius=1.0, center=(0.0, 0.0, 0.0)):
    """Sphere from a regular icosahedron refined `levels` times: 20*4**levels triangles.

    Returns (vertices [nv,3] float64, triangles [nt,3] int32), triangles CCW
    from outside.
    """
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, g, 0], [1, g, 0], [-1, -g, 0], [1, -g, 0],
                  [0, -1, g], [0, 1, g], [0, -1, -g], [0, 1, -g],
                  [g, 0, -1], [g, 0, 1], [-g, 0, -1], [-g, 0, 1]], dtype=np.float64)
    v *= radius / np.linalg.norm(v[0])
    t = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    t = _orient_outward(v, t)
    v, t = _refine(v, t, levels, radius)
    return v + np.asarray(center, dtype=np.float64), t


def ellipsoid(levels, axes=(1.0, 1.0, 1.0), center=(0.0, 0.0, 0.0)):
    """Ellipsoid with the given semi-axes: a unit icosphere scaled along x, y, z (positive
    factors keep the outward orientation)."""
    v, t = icosphere(levels)
    return v * np.asarray(axes, dtype=np.float64) + np.asarray(center, dtype=np.float64), t


def octasphere(levels, radius=1.0, center=(0.0, 0.0, 0.0)):
    """Sphere from a regular octahedron refined `levels` times: 8*4**levels triangles."""
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float64) * radius
    t = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int32)
    t = _orient_outward(v, t)
    v, t = _refine(v, t, levels, radius)
    return v + np.asarray(center, dtype=np.float64), t


def evans_fung_cell(levels, r=3.91, c0=0.81, c2=7.83, c4=-4.39):
    """Biconcave red-blood-cell surface (Evans-Fung map applied to an octahedral sphere).

    A unit-sphere vertex (x, y, z) maps to (r x, r y, +/- z(rho)) with
    rho = r*sqrt(x^2+y^2) and z(rho) = 1/2 sqrt(1-(rho/r)^2) (c0 + c2 (rho/r)^2 + c4 (rho/r)^4),
    the sign taken from the sphere vertex's z. Units are micrometres.
    """
    v, t = octasphere(levels, 1.0)
    s2 = np.clip(v[:, 0] ** 2 + v[:, 1] ** 2, 0.0, 1.0)
    zabs = 0.5 * np.sqrt(1.0 - s2) * (c0 + c2 * s2 + c4 * s2 * s2)
    out = np.empty_like(v)
    out[:, 0] = r * v[:, 0]
    out[:, 1] = r * v[:, 1]
    out[:, 2] = np.where(v[:, 2] >= 0.0, zabs, -zabs)
    return out, t


def _random_rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def place_cells(v, t, n_cells, box=40.0, min_gap=0.5, seed=0, max_tries=100000):
    """Copies of one surface, each randomly rotated (uniform quaternion) and shifted
    to a centre drawn uniformly in [0, box]^3, rejected while any vertex comes
    closer than `min_gap` to a vertex of an already placed copy.
    Returns (vertices, triangles, body_of_panel)."""
    rng = np.random.default_rng(seed)
    verts, tris, body = [], [], []
    placed = []
    off = 0
    for c in range(n_cells):
        for _ in range(max_tries):
            rv = v @ _random_rotation(rng).T + rng.uniform(0.0, box, size=3)
            ok = True
            for pv in placed:
                lo = np.maximum(rv.min(0), pv.min(0)) - min_gap
                hi = np.minimum(rv.max(0), pv.max(0)) + min_gap
                if np.any(lo > hi):
                    continue
                d2 = ((rv[:, None, :] - pv[None, :, :]) ** 2).sum(-1)
                if d2.min() < min_gap * min_gap:
                    ok = False
                    break
            if ok:
                break
        else:
            raise RuntimeError("could not place cell %d" % c)
        placed.append(rv)
        verts.append(rv)
        tris.append(t + off)
        body.append(np.full(len(t), c, dtype=np.int32))
        off += len(rv)
    return np.concatenate(verts), np.concatenate(tris).astype(np.int32), np.concatenate(body)


def random_vector(n, seed=0):
    """Seeded standard-normal vector of length n (float64)."""
    return np.random.default_rng(seed).standard_normal(n)


def point_charge_dirichlet(points, z0=(0.0, 0.0, 3.0)):
    """Potential of a unit point charge at z0 at the given points: 1/(4 pi |x - z0|)."""
    d = np.asarray(points, dtype=np.float64) - np.asarray(z0, dtype=np.float64)
    return 1.0 / (4.0 * np.pi * np.sqrt((d * d).sum(-1)))


def smooth_random_field(points, seed=0, modes=8, k_min=1.0, k_max=3.0):
    """Seeded smooth vector field at the given points: a sum of `modes` plane waves
    a_m sin(k_m . x + phase_m) with random unit amplitudes a_m (3-vectors), wave vectors of
    length in [k_min, k_max] and phases. Boundary data that excites many spherical harmonics at
    once (unlike a rigid motion of a sphere, which is an eigenfunction of its layer operators)."""
    rng = np.random.default_rng(seed)
    x = np.asarray(points, dtype=np.float64)
    out = np.zeros((len(x), 3))
    for _ in range(modes):
        k = rng.standard_normal(3)
        k *= rng.uniform(k_min, k_max) / np.linalg.norm(k)
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        out += a[None, :] * np.sin(x @ k + rng.uniform(0.0, 2.0 * np.pi))[:, None]
    return out
