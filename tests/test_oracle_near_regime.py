"""Pins for the oracle's near-singular regime (Sec. 2.3, eqs. gauss:1st-kind and
gauss:2nd-kind): a panel j whose centroid lies within 2 sqrt(2 S_j) of the
collocation point c_i is integrated with the 20-point rule, a farther panel with
the K-point rule.

Each oracle entry is compared with the exact integral, taken here by an
independent route: the source panel is split into 4^L congruent triangles and
each is integrated with a collapsed n x n Gauss-Legendre product (numpy's
leggauss nodes, not the oracle's), converged to ~1e-14. Then:
  - entries just inside the radius agree with the exact integral to the accuracy
    of a degree-7 rule, entries just outside only to that of the K-point rule;
  - the accuracy jumps at exactly the stated radius, located by bisection along
    several directions, and the radius is measured with the SOURCE panel's area
    S_j: the target panels are made 400 times smaller and 25 times larger than
    the source, which would move the jump by factors 20 and 5 if S_i were used;
  - the same holds on the rows of a refined and of a randomly skewed icosphere,
    whose neighbouring panels differ in area.
"""
import numpy as np
import pytest

from oracle import dense
from synth import icosphere

NEAR_FACTOR = 2.0


def _exact(P, c, kind, L=4, n=10):
    """Integral over triangle P (3 x 3) of the kernel at the point c, by 4^L subdivision and
    an n x n collapsed Gauss product per sub-triangle. Returns a scalar (Laplace) or 3 x 3."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    tris = [np.asarray(P, dtype=np.float64)]
    for _ in range(L):
        nxt = []
        for a, b, cc in tris:
            ab, bc, ca = 0.5 * (a + b), 0.5 * (b + cc), 0.5 * (cc + a)
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, cc]), np.array([ab, bc, ca])]
        tris = nxt
    T = np.array(tris)  # [m, 3, 3]
    a, b, cc = T[:, 0], T[:, 1], T[:, 2]
    jac = np.linalg.norm(np.cross(b - a, cc - a), axis=1)  # twice each sub-triangle's area
    U, Vv = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    u, v, wq = U.ravel(), Vv.ravel(), (WU * WV * U).ravel()
    # y = a + u (b - a) + u v (c - b): the unit square onto the triangle, Jacobian u * jac
    y = a[:, None, :] + u[None, :, None] * (b - a)[:, None, :] + (u * v)[None, :, None] * (cc - b)[:, None, :]
    d = np.asarray(c)[None, None, :] - y  # collocation point minus integration point
    r = np.linalg.norm(d, axis=2)
    W = wq[None, :] * jac[:, None]
    e1, e2 = P[1] - P[0], P[2] - P[0]
    nrm = np.cross(e1, e2)
    nrm = nrm / np.linalg.norm(nrm)
    if kind == "lsl":
        return np.sum(W / r) / (4.0 * np.pi)
    if kind == "ldl":
        return np.sum(W * (d @ nrm) / r ** 3) / (4.0 * np.pi)
    if kind == "ssl":  # Stokeslet, mu = 1: -1/(8 pi) int (I/r + d d^T / r^3)
        G = np.eye(3)[None, None] / r[..., None, None] + d[..., :, None] * d[..., None, :] / r[..., None, None] ** 3
        return -np.einsum("mk,mkab->ab", W, G) / (8.0 * np.pi)
    if kind == "sdl":  # stresslet: 1/(8 pi) int 6 e e^T (e.n)/r^5, e = y - c = -d
        en = -(d @ nrm)
        T5 = 6.0 * d[..., :, None] * d[..., None, :] * en[..., None, None] / r[..., None, None] ** 5
        return np.einsum("mk,mkab->ab", W, T5) / (8.0 * np.pi)
    raise ValueError(kind)


def _oracle_entry(P, Q, kind):
    """The oracle's (target Q's centroid, source P) entry, from a two-panel mesh [Q, P]."""
    v = np.vstack([Q, P])
    t = np.array([[0, 1, 2], [3, 4, 5]])
    if kind in ("lsl", "ldl"):
        M = dense.Mesh(v, t, k=4, near_factor=NEAR_FACTOR)
        return M.laplace_matrix(kind="sl" if kind == "lsl" else "dl", rows=[0])[0, 1]
    M = dense.Mesh(v, t, k=3, near_factor=NEAR_FACTOR)
    A = M.stokes_matrix(kind="sl" if kind == "ssl" else "dl", mu=1.0, rows=[0])
    return A[:, 3:6]


def _rel_err(P, Q, kind):
    c = Q.mean(0)
    ex = _exact(P, c, kind)
    got = _oracle_entry(P, Q, kind)
    return float(np.linalg.norm(np.atleast_1d(got - ex)) / np.linalg.norm(np.atleast_1d(ex)))


def _area(P):
    return 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))


def _target_panel(centre, area, rng):
    """A random triangle of the given area with its centroid at `centre`."""
    while True:
        T = rng.standard_normal((3, 3))
        if _area(T) > 0.2:
            break
    T = T - T.mean(0)
    return centre + T * np.sqrt(area / _area(T))


def _source_panels():
    rng = np.random.default_rng(7)
    out = [np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.8, 0.0]])]  # skewed, in z = 0
    while len(out) < 4:  # random, obtuse or thin allowed but not degenerate
        P = rng.standard_normal((3, 3))
        e = [np.linalg.norm(P[(k + 1) % 3] - P[k]) for k in range(3)]
        if _area(P) > 0.08 * max(e) ** 2:
            out.append(P)
    return out


# (kind, whether the direction may lie in the source plane (the double layers vanish there),
# accuracy of the 20-point rule just inside the radius on these panels: the stresslet's
# stronger singularity and the thin random panel give the larger figures)
CASES = [("lsl", True, 5e-6), ("ldl", False, 5e-5), ("ssl", True, 2e-5), ("sdl", False, 2e-4)]


@pytest.mark.parametrize("kind,in_plane_ok,near_acc", CASES)
def test_near_rule_switches_at_two_sqrt_two_source_area(kind, in_plane_ok, near_acc):
    rng = np.random.default_rng({"lsl": 1, "ldl": 2, "ssl": 3, "sdl": 4}[kind])
    for P in _source_panels():
        Sj = _area(P)
        R = NEAR_FACTOR * np.sqrt(2.0 * Sj)
        cj = P.mean(0)
        nrm = np.cross(P[1] - P[0], P[2] - P[0])
        nrm /= np.linalg.norm(nrm)
        dirs = []
        while len(dirs) < 3:
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            if not in_plane_ok and abs(u @ nrm) < 0.3:
                continue
            dirs.append(u)
        for u in dirs:
            for ratio in (1.0 / 400.0, 25.0):  # target area S_i = ratio * S_j
                Q0 = _target_panel(np.zeros(3), ratio * Sj, rng)

                def err(s):
                    return _rel_err(P, cj + s * R * u + Q0, kind)

                e_in, e_out = err(0.97), err(1.03)
                # inside: the 20-point (degree-7) rule; outside: the K-point rule
                assert e_in < near_acc, (kind, e_in)
                assert e_out < 2e-2, (kind, e_out)
                assert e_out > 20.0 * e_in, (kind, e_in, e_out)
                # the jump sits at s = 1 (distance 2 sqrt(2 S_j) from the source centroid)
                thr = np.sqrt(e_in * e_out)
                lo, hi = 0.97, 1.03
                for _ in range(14):
                    mid = 0.5 * (lo + hi)
                    if err(mid) < thr:
                        lo = mid
                    else:
                        hi = mid
                assert abs(0.5 * (lo + hi) - 1.0) < 1e-3, (kind, lo, hi)


def _mesh_pair_errors(v, t, band=(0.85, 1.2)):
    """Errors of single-layer oracle entries for all panel pairs whose centroid distance lies
    within `band` times the source radius 2 sqrt(2 S_j). Returns (errors, d/R_j, d/R_i)."""
    M = dense.Mesh(v, t, k=4, near_factor=NEAR_FACTOR)
    P = v[t]
    c = P.mean(1)
    S = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    R = NEAR_FACTOR * np.sqrt(2.0 * S)
    rng = np.random.default_rng(11)
    rows = rng.choice(len(t), size=24, replace=False)
    A = M.laplace_matrix(rows=rows)
    errs, sj, si = [], [], []
    for r, i in enumerate(rows):
        d = np.linalg.norm(c - c[i], axis=1)
        for j in np.nonzero((d > band[0] * R) & (d < band[1] * R))[0]:
            if j == i:
                continue
            ex = _exact(P[j], c[i], "lsl", L=3)
            errs.append(abs(A[r, j] - ex) / ex)
            sj.append(d[j] / R[j])
            si.append(d[j] / R[i])
    return np.array(errs), np.array(sj), np.array(si)


@pytest.mark.parametrize("skew", [0.0, 0.25])
def test_near_regime_on_mesh_rows(skew):
    v, t = icosphere(3)
    if skew:
        rng = np.random.default_rng(5)
        v = v * (1.0 + skew * rng.uniform(-1, 1, size=(len(v), 1)))  # panels of unequal area
    err, sj, si = _mesh_pair_errors(v, t)
    inside, outside = sj < 1.0, sj > 1.0
    assert inside.sum() > 20 and outside.sum() > 20
    # the 20-point rule inside, the 4-point rule outside: typical errors two orders apart
    assert err[inside].max() < 1e-5
    assert np.median(err[outside]) > 100.0 * np.median(err[inside])
    if skew:
        # pairs that the target's own radius would classify the other way
        flip_in = inside & (si > 1.0)
        flip_out = outside & (si < 1.0)
        assert flip_in.sum() > 20 and flip_out.sum() > 20
        assert err[flip_in].max() < 1e-5
        assert np.median(err[flip_out]) > 100.0 * np.median(err[flip_in])
