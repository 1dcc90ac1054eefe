"""Dense collocation BEM operators (oracle; test infrastructure only).

Thin ctypes front end over oracle/csrc/oracle_bem.c, which evaluates rows of
the dense matrices by the paper's mat-vec loop (Appendix, Algorithm
"Matrix-vector multiplication") with the three integration regimes of Sec. 2.3.

Operators (all FP64):
  laplace_sl : V_ij = 1/(4 pi) int_j 1/r dS          (eq. laplace_bem_G with G = 1/(4 pi r))
  laplace_dl : K_ij = 1/(4 pi) int_j n_j.(c_i-y)/r^3 dS (eq. laplace_bem_dGdn)
  stokes_sl  : A_iJ = -1/(8 pi mu) int_J G dS          (eqs. stokes_bem_discretized, stokeslet)
  stokes_dl  : B_iJ = 1/(8 pi) int_J T_abk n_k dS      (eq. stresslet, read as T contracted once with n)

Pins (tests/test_oracle_bem.py): V 1 -> 1 on the unit sphere; V z ~ z/3
(eigenvalue 1/(2n+1)); K 1 = -1/2 (Gauss identity); (1/8pi) int T n = +1/2 I;
closed-form self-integral of an equilateral triangle; trace identity of the
Stokes self block; brute-force Duffy quadrature of the self-integrals;
Laplace solve error vs the analytic flux falling with N; Stokes drag vs
6 pi mu a U. The near-singular regime (the 2 sqrt(2 S_j) switch and the
20-point rule) is pinned against an independent quadrature of each entry in
tests/test_oracle_near_regime.py.
"""
import ctypes
import numpy as np

from . import build as _build
from .panels import panel_vertices
from .quadrature import triangle_rule, near_rule

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        for name in ("oracle_laplace_rows", "oracle_stokes_rows"):
            getattr(L, name).restype = None
        L.oracle_self_integrals.restype = None
        L.oracle_nbody_laplace.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


class Mesh:
    """Panels plus the far and near rules used by every oracle operator."""

    def __init__(self, vertices, triangles, k=4, near_factor=2.0, near_k=20):
        self.pv = panel_vertices(vertices, triangles)
        self.n = len(self.pv)
        self.k = k
        fb, fw = triangle_rule(k)
        # near rule: a collapsed Gauss product of nu x (nu - 1) points (5 x 4 = 20 by default,
        # the K ~ 20 of Sec. 2.3); other point counts name a plain triangle rule
        nu = int(round((1.0 + np.sqrt(1.0 + 4.0 * near_k)) / 2.0))
        if nu * (nu - 1) == near_k and 3 <= nu <= 7:
            nb, nw = near_rule(nu, nu - 1)
        else:
            nb, nw = triangle_rule(near_k)
        self.fb, self.fw = np.ascontiguousarray(fb), np.ascontiguousarray(fw)
        self.nb, self.nw = np.ascontiguousarray(nb), np.ascontiguousarray(nw)
        self.near_factor = float(near_factor)

    def _common(self):
        return (ctypes.c_int(self.n), _ptr(self.pv), ctypes.c_int(len(self.fw)), _ptr(self.fb), _ptr(self.fw),
                ctypes.c_int(len(self.nw)), _ptr(self.nb), _ptr(self.nw), ctypes.c_double(self.near_factor))

    def _rows(self, rows):
        if rows is None:
            rows = np.arange(self.n, dtype=np.int64)
        return np.ascontiguousarray(np.asarray(rows, dtype=np.int64))

    def laplace_apply(self, x, kind="sl", rows=None):
        """(A x)[rows] for the Laplace single (sl) or double (dl) layer."""
        rows = self._rows(rows)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(len(rows))
        lib().oracle_laplace_rows(*self._common(), ctypes.c_int(0 if kind == "sl" else 1),
                                  ctypes.c_int(len(rows)), rows.ctypes.data_as(_ip), _ptr(x), _ptr(y), None)
        return y

    def laplace_matrix(self, kind="sl", rows=None):
        rows = self._rows(rows)
        A = np.zeros((len(rows), self.n))
        lib().oracle_laplace_rows(*self._common(), ctypes.c_int(0 if kind == "sl" else 1),
                                  ctypes.c_int(len(rows)), rows.ctypes.data_as(_ip), None, None, _ptr(A))
        return A

    def stokes_apply(self, x, kind="sl", mu=1.0, rows=None):
        """(A x)[rows] with x laid out [n, 3]; returns [len(rows), 3]."""
        rows = self._rows(rows)
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
        y = np.zeros(3 * len(rows))
        lib().oracle_stokes_rows(*self._common(), ctypes.c_int(0 if kind == "sl" else 1), ctypes.c_double(mu),
                                 ctypes.c_int(len(rows)), rows.ctypes.data_as(_ip), _ptr(x), _ptr(y), None)
        return y.reshape(-1, 3)

    def stokes_matrix(self, kind="sl", mu=1.0, rows=None):
        rows = self._rows(rows)
        A = np.zeros((3 * len(rows), 3 * self.n))
        lib().oracle_stokes_rows(*self._common(), ctypes.c_int(0 if kind == "sl" else 1), ctypes.c_double(mu),
                                 ctypes.c_int(len(rows)), rows.ctypes.data_as(_ip), None, None, _ptr(A))
        return A


def self_integrals(v9, c):
    """(int 1/|c-y| dS, int d d^T/|d|^3 dS) over one flat panel, c inside it."""
    v9 = np.ascontiguousarray(v9, dtype=np.float64).reshape(9)
    c = np.ascontiguousarray(c, dtype=np.float64).reshape(3)
    I1 = ctypes.c_double(0.0)
    D = np.zeros(9)
    lib().oracle_self_integrals(_ptr(v9), _ptr(c), ctypes.byref(I1), _ptr(D))
    return I1.value, D.reshape(3, 3)


def nbody_laplace(targets, sources, q, grad=False):
    """Direct sums phi_i = sum_j q_j/|x_i - y_j| (and the gradient) in FP64."""
    t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    phi = np.zeros(len(t))
    g = np.zeros((len(t), 3)) if grad else None
    lib().oracle_nbody_laplace(ctypes.c_int(len(t)), _ptr(t), ctypes.c_int(len(s)), _ptr(s), _ptr(q),
                               _ptr(phi), _ptr(g))
    return (phi, g) if grad else phi
