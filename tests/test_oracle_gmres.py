"""Pins for the oracle's GMRES: dense LU (library routine), finite termination,
monotone residual estimates, and the BEM system itself."""
import numpy as np

from oracle import dense, panels
from oracle.gmres import gmres
from synth import icosphere, point_charge_dirichlet


def test_gmres_matches_lu_random():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, it, hist = gmres(lambda v, k: A @ v, b, tol=1e-13, restart=n, max_iter=n)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
    assert hist[-1] <= 1e-13


def test_gmres_finite_termination():
    rng = np.random.default_rng(3)
    n = 12
    A = rng.standard_normal((n, n)) + 5 * np.eye(n)
    b = rng.standard_normal(n)
    x, it, hist = gmres(lambda v, k: A @ v, b, tol=1e-30, restart=n, max_iter=n)
    assert it == n
    assert np.linalg.norm(A @ x - b) < 1e-10 * np.linalg.norm(b)


def test_gmres_restarted_converges():
    rng = np.random.default_rng(1)
    n = 80
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, it, hist = gmres(lambda v, k: A @ v, b, tol=1e-10, restart=8, max_iter=400)
    assert np.linalg.norm(A @ x - b) <= 2e-10 * np.linalg.norm(b)
    assert it > 8


def test_gmres_bem_system():
    v, t = icosphere(2)
    M = dense.Mesh(v, t, k=4)
    c, _, _ = panels.geometry(v, t)
    phi = point_charge_dirichlet(c)
    b = 0.5 * phi + M.laplace_apply(phi, kind="dl")
    V = M.laplace_matrix()
    x, it, hist = gmres(lambda u, k: M.laplace_apply(u), b, tol=1e-12, restart=50, max_iter=200)
    assert np.linalg.norm(x - np.linalg.solve(V, b)) < 1e-9 * np.linalg.norm(x)
