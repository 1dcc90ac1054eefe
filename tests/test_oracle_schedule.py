"""Pins for the relaxation schedule (eqs. matrix-perturbation and fmm_p) and the
Richardson utility (Sec. 3.3) against hand-computed and printed values."""
import pytest

from oracle import richardson
from oracle.schedule import epsilon, order_from_epsilon, relaxed_p, schedule
from tests.golden.values import paper_values


def test_epsilon_definition():
    assert epsilon(1e-6, 1.0) == 1e-6
    assert epsilon(1e-6, 5.0) == 1e-6          # min(||r||, 1) caps the residual at 1
    assert epsilon(1e-6, 1e-3) == pytest.approx(1e-3)
    assert epsilon(1e-6, 1e-7) == 1.0          # never above 1


def test_order_hand_values():
    # ceil(-log2 eps): 1e-3 -> 9.97 -> 10; 5e-4 -> 10.97 -> 11; 0.1 -> 3.32 -> 4; 1e-6 -> 19.93 -> 20
    assert order_from_epsilon(1e-3) == 10
    assert order_from_epsilon(5e-4) == 11
    assert order_from_epsilon(0.1) == 4
    assert order_from_epsilon(1e-6) == 20
    # exact powers of two sit on the boundary: -log2(2^-k) = k
    for k in range(1, 30):
        assert order_from_epsilon(2.0 ** -k) == k
    assert order_from_epsilon(0.5 + 1e-16) == 1
    assert order_from_epsilon(1.0) == 0


def test_relaxed_p_clamps():
    assert relaxed_p(1e-6, 1.0, 10, 3) == 10     # first step: p_initial
    assert relaxed_p(1e-6, 1e-3, 12, 3) == 10
    assert relaxed_p(1e-6, 1e-5, 12, 3) == 4
    assert relaxed_p(1e-6, 1e-6, 12, 3) == 3     # eps = 1 -> 0 -> p_min
    assert relaxed_p(1e-5, 1e-3, 16, 5) == 7


def test_schedule_sequence():
    rhos = [1.0, 0.3, 1e-2, 1e-3, 1e-4, 1e-5, 3e-6]
    assert schedule(1e-6, rhos, 12, 3) == [12, 12, 12, 10, 7, 4, 3]


def test_richardson_paper_example():
    # The printed drags are rounded to 3 decimals, so they fix the observed order
    # only up to that rounding: the printed order 0.52 must lie inside the range of
    # orders reachable within +-0.0005 of each printed value (c = 4).
    import itertools
    pv = paper_values()
    f = [pv["rbc_fx_512"], pv["rbc_fx_2048"], pv["rbc_fx_8192"]]
    orders = [richardson.observed_order(f[0] + a, f[1] + b, f[2] + c, 4.0)
              for a, b, c in itertools.product((-5e-4, 5e-4), repeat=3)]
    assert min(orders) < pv["rbc_observed_order"] < max(orders)
    assert max(orders) - min(orders) < 0.4
    fbar = richardson.extrapolate(*f)
    assert fbar < f[2] < f[1] < f[0]  # a monotone sequence extrapolates beyond its finest value
    # an exactly geometric sequence of differences recovers its order and limit
    g = [1.0 - 4.0 ** -0.5 * k for k in (1.0, 0.5, 0.25)]
    assert abs(richardson.observed_order(g[0], g[1], g[2], 4.0) - 0.5) < 1e-12
