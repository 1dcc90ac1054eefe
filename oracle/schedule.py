"""Relaxation schedule for the expansion order p (oracle; test infrastructure only).

eq. matrix-perturbation: eps_k = min(eta / min(||r_{k-1}||, 1), 1), with the
residual read as the relative residual rho = ||r|| / ||b|| (rho_0 = 1);
eq. fmm_p: p ~ ceil(-log2 eps), clamped to [p_min, p_initial] (p_min as in
Table stokes_min_p).

ceil(-log2 eps) is taken exactly: with eps = f 2^e, f in [0.5, 1) (frexp),
-log2 eps lies in (-e, 1 - e], so the ceiling is 1 - e. The CUDA path makes the
same decision in the same precision.
Pinned by hand-computed sequences (tests/test_oracle_schedule.py).
"""
import math


def epsilon(eta, rho_prev):
    return min(eta / min(rho_prev, 1.0), 1.0)


def order_from_epsilon(eps):
    if eps >= 1.0:
        return 0
    _, e = math.frexp(eps)
    return 1 - e


def relaxed_p(eta, rho_prev, p_initial, p_min):
    p = order_from_epsilon(epsilon(eta, rho_prev))
    return min(p_initial, max(p_min, p))


def schedule(eta, rhos, p_initial, p_min):
    """p_k for k = 1.. given the residuals rho_0 = 1, rho_1, ... that precede each step."""
    return [relaxed_p(eta, r, p_initial, p_min) for r in rhos]
