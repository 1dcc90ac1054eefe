"""Textbook restarted GMRES(m) (Saad & Schultz 1986; the solver of Sec. 2.4).

Oracle; test infrastructure only. Modified Gram-Schmidt Arnoldi, Givens
rotations on the Hessenberg matrix, x0 = 0 by default, stop when the GMRES
residual estimate |g_{k+1}| / ||b|| <= tol or after max_iter Arnoldi steps.
At each restart the true residual b - A x is recomputed.

`matvec(v, k)` receives the running Arnoldi step count k (0-based) so that a
caller can model an inexact product; the oracle's own operators ignore it.
Pinned by: agreement with a dense LU solve (numpy.linalg.solve) on small
systems, exact termination in n steps for an n x n system, and a monotone
residual history (tests/test_oracle_gmres.py).
"""
import numpy as np


def gmres(matvec, b, tol=1e-6, restart=50, max_iter=100, x0=None):
    b = np.asarray(b, dtype=np.float64)
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    r = b - (matvec(x, it) if np.any(x) else 0.0)
    beta = np.linalg.norm(r)
    hist.append(beta / bnorm)
    while hist[-1] > tol and it < max_iter:
        m = min(restart, max_iter - it)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            w = matvec(V[k], it)
            it += 1
            for j in range(k + 1):
                H[j, k] = np.dot(V[j], w)
                w = w - H[j, k] * V[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for j in range(k):
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            hist.append(abs(g[k + 1]) / bnorm)
            k_done = k + 1
            if hist[-1] <= tol or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + V[:k_done].T @ y
        if hist[-1] <= tol or it >= max_iter:
            break
        r = b - matvec(x, it)
        beta = np.linalg.norm(r)
        hist[-1] = beta / bnorm
    return x, it, hist
