"""The harmonic decomposition behind the FMM stresslet double layer (eq. stresslet), checked
against the direct sum on random sources (no GPU).

With r = x - y, dipole moments m^(j) = a_j n + n_j a (j = 1, 2, 3) and m^(0) = (a.y) n + (n.y) a,
and S_j(x) = sum_s m^(j).(x - y) / |x - y|^3 (dipole potentials),

    sum_s (a.r)(n.r) r_i / |r|^5 = -(1/6) [ x_j d_i S_j - d_i S_0 - S_i ],

so the stresslet sum takes four Laplace dipole expansions and the Stokeslet's evaluation
u_i = phi_i - x_j d_i phi_j + d_i phi_0 (with phi = S): the FMM double layer is that
evaluation times -1/(8 pi) (the operator's 1/(8 pi) times the kernel's 6 (e.u)(e.n) e / r^5
with e = -r)."""
import numpy as np


def _dipole(m, y, x):
    """phi(x) = sum m.(x - y)/|x - y|^3 and its gradient, for moments m [S,3] at y [S,3]."""
    r = x[None, :] - y
    d = np.linalg.norm(r, axis=1)
    mr = (m * r).sum(1)
    phi = np.sum(mr / d ** 3)
    grad = np.sum(m / d[:, None] ** 3 - 3.0 * (mr / d ** 5)[:, None] * r, axis=0)
    return phi, grad


def test_stresslet_sum_equals_four_dipole_potentials():
    rng = np.random.default_rng(0)
    S = 40
    y = rng.standard_normal((S, 3))
    a = rng.standard_normal((S, 3))
    n = rng.standard_normal((S, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    for x in (np.array([4.0, -1.0, 2.5]), np.array([-3.0, 3.0, 3.0]), 0.1 * rng.standard_normal(3) + 5.0):
        r = x[None, :] - y
        d = np.linalg.norm(r, axis=1)
        direct = np.sum(((a * r).sum(1) * (n * r).sum(1) / d ** 5)[:, None] * r, axis=0)
        phis, grads = [], []
        for j in range(3):
            m = a[:, j:j + 1] * n + n[:, j:j + 1] * a
            f, g = _dipole(m, y, x)
            phis.append(f)
            grads.append(g)
        m0 = (a * y).sum(1)[:, None] * n + (n * y).sum(1)[:, None] * a
        f0, g0 = _dipole(m0, y, x)
        # Stokeslet-form evaluation u_i = S_i - x_j d_i S_j + d_i S_0
        u = np.array([phis[i] - sum(x[j] * grads[j][i] for j in range(3)) + g0[i] for i in range(3)])
        assert np.allclose(direct, u / 6.0, rtol=1e-12, atol=1e-14 * np.abs(direct).max())
        # a plausible slip (dropping S_0 or the S_i term) breaks it
        assert not np.allclose(direct, (u - np.array(g0)) / 6.0, rtol=1e-6)
