"""Quadrature rules on a triangle (oracle; test infrastructure only).

The paper gives only the number of points: K = 4 (Laplace) or 3 (Stokes) for
far panels and K ~ 20 for near-singular panels (Sec. 2.3, eqs. gauss:1st-kind,
gauss:2nd-kind). Weights are area-normalised (sum to 1), matching the q_k of
those equations. Rules, written from their published definitions:

  K = 1 : centroid (degree 1).
  K = 3 : interior Strang-Fix rule (2/3, 1/6, 1/6) and permutations, q = 1/3 (degree 2).
  K = 4 : Strang-Fix / Dunavant degree-3 rule: centroid with q = -27/48 and
          (3/5, 1/5, 1/5) and permutations with q = 25/48.
  K = 7 : Radon degree-5 rule.
  near  : collapsed (Duffy) product rule, 5 Gauss-Legendre nodes in the
          collapsed direction u (Jacobian u folded into the weight) times 4
          nodes in v: 20 points, exact to total degree 7.

Gauss-Legendre nodes come from the Golub-Welsch eigenvalue method.
Pinned by: exact integration of every monomial up to the rule's degree
(closed form 2 a! b! / (a+b+2)! for the area-normalised integral of
lambda_2^a lambda_3^b), tests/test_oracle_quadrature.py.
"""
import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1] (nodes, weights summing to 1), Golub-Welsch."""
    k = np.arange(1, n)
    beta = k / np.sqrt(4.0 * k * k - 1.0)
    J = np.diag(beta, 1) + np.diag(beta, -1)
    x, V = np.linalg.eigh(J)
    w = 2.0 * V[0, :] ** 2
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(k):
    """Barycentric points [k, 3] and area-normalised weights [k] of a K-point rule."""
    if k == 1:
        return np.array([[1 / 3, 1 / 3, 1 / 3]]), np.array([1.0])
    if k == 3:
        a, b = 2.0 / 3.0, 1.0 / 6.0
        return np.array([[a, b, b], [b, a, b], [b, b, a]]), np.full(3, 1.0 / 3.0)
    if k == 4:
        a, b = 0.6, 0.2
        return (np.array([[1 / 3, 1 / 3, 1 / 3], [a, b, b], [b, a, b], [b, b, a]]),
                np.array([-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0]))
    if k == 7:
        s = np.sqrt(15.0)
        a1 = (6.0 - s) / 21.0
        a2 = (6.0 + s) / 21.0
        w1 = (155.0 - s) / 1200.0
        w2 = (155.0 + s) / 1200.0
        pts = [[1 / 3, 1 / 3, 1 / 3]]
        wts = [9.0 / 40.0]
        for a, w in ((a1, w1), (a2, w2)):
            b = 1.0 - 2.0 * a
            pts += [[b, a, a], [a, b, a], [a, a, b]]
            wts += [w, w, w]
        return np.array(pts), np.array(wts)
    raise ValueError("no %d-point triangle rule" % k)


def near_rule(nu=5, nv=4):
    """Collapsed product rule: lambda_1 = 1 - u, lambda_2 = u (1 - v), lambda_3 = u v.

    The area-normalised integral is 2 int_0^1 int_0^1 f u du dv; the factor u
    is folded into the weights. Returns (barycentric [nu*nv, 3], weights)."""
    xu, wu = gauss_legendre(nu)
    xv, wv = gauss_legendre(nv)
    pts, wts = [], []
    for i in range(nu):
        for j in range(nv):
            u, v = xu[i], xv[j]
            pts.append([1.0 - u, u * (1.0 - v), u * v])
            wts.append(2.0 * wu[i] * wv[j] * u)
    return np.array(pts), np.array(wts)


def rule_degree(k):
    """Total degree integrated exactly: the triangle rules, and the collapsed near rules of
    nu x (nu - 1) points (degree 2 (nu - 1) - 1 from the nu - 1 nodes in v)."""
    return {1: 1, 3: 2, 4: 3, 7: 5, 6: 3, 12: 5, 20: 7, 30: 9, 42: 11}[k]
