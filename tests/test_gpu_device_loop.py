"""The device-resident GMRES cycle (fmmbem_set_device_loop) against the host loop, through
the C ABI.

Both run the same steps (Sec. 2.4 and 2.6): the same mat-vec kernels at the same orders, the
same Arnoldi kernel and the same FP64 column update, done by one device thread instead of the
host. What the comparison can hold them to depends on the arithmetic:
  - FP64 solves: the mat-vec varies between runs only at rounding level (FP64 atomics), so
    the two loops take the same steps at the same orders, with residual estimates within 1e-5
    and solutions within 1e-7 relative (GMRES amplifies the rounding in its late steps);
  - mixed-precision solves: the FP32 passes add partial results with atomics in an order that
    varies from run to run (about 1e-7 relative per mat-vec, amplified by GMRES), so two solves
    of one system differ at that level whichever loop runs them. The device loop's orders are
    checked against the relaxation rule applied to its own residual history (exact: the rule
    is frexp of a ratio), its step count against the host loop's (within one), and its solution
    against the host loop's (1e-5 relative) and the oracle (residual <= 2 tol).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05957_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def sphere1280(torch_cuda):
    from oracle import dense, panels
    from synth import icosphere, point_charge_dirichlet
    v, t = icosphere(3)
    M = dense.Mesh(v, t, k=4)
    c, _, _ = panels.geometry(v, t)
    phi = point_charge_dirichlet(c)
    b = 0.5 * phi + M.laplace_apply(phi, kind="dl")
    return dict(v=v, t=t, b=b, A=M.laplace_matrix())


def _solve(torch, v, t, b, device_loop, repeat=1, solve_kw=None, **kw):
    from paper_1506_05957_gb300 import FmmBem
    h = FmmBem(v, t, gauss_k=4, ncrit=150, theta=0.5, **kw)
    if device_loop:
        h.set_device_loop(True)
    out = []
    for _ in range(repeat):
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        r = h.solve(torch.tensor(b, dtype=torch.float64, device="cuda"), x, **(solve_kw or {}))
        torch.cuda.synchronize()
        out.append((r, x.cpu().numpy()))
    h.close()
    return out


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _orders_follow_rule(r, tol, p_initial, p_min, relax):
    """Step j's order is the relaxation rule at the residual estimate before it (1 at the start)."""
    from paper_1506_05957_gb300 import fmmbem_relaxed_p
    for j, p in enumerate(r["p_hist"]):
        want = fmmbem_relaxed_p(tol, r["res_hist"][j], p_initial, p_min) if relax else p_initial
        assert p == want, (j, p, want)


@pytest.mark.parametrize("precision,restart,relax,max_iter", [
    ("mixed", 50, True, 100),   # one cycle, p relaxed 10 -> 3
    ("mixed", 4, True, 100),    # restarts every four steps
    ("mixed", 50, False, 100),  # fixed p
    ("fp64", 50, True, 100),
    ("fp64", 4, True, 100),
    ("mixed", 50, True, 6),     # stops on the iteration budget, not converged
])
def test_device_loop_matches_host_loop(torch_cuda, sphere1280, precision, restart, relax, max_iter):
    from paper_1506_05957_gb300 import FMMBEM_FP64, FMMBEM_MIXED
    s = sphere1280
    prec = FMMBEM_FP64 if precision == "fp64" else FMMBEM_MIXED
    kw = dict(p_max=10, precision=prec, restart=restart, max_iter=max_iter)
    sk = dict(tol=1e-6, relax=relax, p_initial=10, p_min=3)
    (rh, xh), = _solve(torch_cuda, s["v"], s["t"], s["b"], False, solve_kw=sk, **kw)
    runs = _solve(torch_cuda, s["v"], s["t"], s["b"], True, repeat=2, solve_kw=sk, **kw)
    for rd, xd in runs:  # the second solve replays the graph built by the first
        _orders_follow_rule(rd, sk["tol"], sk["p_initial"], sk["p_min"], relax)
        assert rd["converged"] == rh["converged"]
        if precision == "fp64":
            assert rd["iters"] == rh["iters"] and rd["p_hist"] == rh["p_hist"]
            np.testing.assert_allclose(rd["res_hist"], rh["res_hist"], rtol=1e-5, atol=0)
            assert _rel(xd, xh) < 1e-7
        else:
            assert abs(rd["iters"] - rh["iters"]) <= 1
            if max_iter != 6:
                assert _rel(xd, xh) < 1e-5
    if max_iter == 6:
        assert not rh["converged"] and rh["iters"] == 6 and all(r["iters"] == 6 for r, _ in runs)
    else:
        assert rh["converged"]
        for _, xd in runs:
            r_or = np.linalg.norm(s["A"] @ xd - s["b"]) / np.linalg.norm(s["b"])
            assert r_or <= 2e-6


def test_device_loop_stokes(torch_cuda):
    """Stokes flow around four red blood cells (four expansions per cell, the vector near field)
    through the device cycle: uniform flow, tol 1e-6, p 16 -> 4."""
    from paper_1506_05957_gb300 import FmmBem, FMMBEM_MIXED, FMMBEM_STOKES
    from synth import evans_fung_cell, place_cells
    torch = torch_cuda
    cv, ct = evans_fung_cell(4)
    v, t, _ = place_cells(cv, ct, 4, box=40.0, min_gap=0.5, seed=1016323256)
    sk = dict(tol=1e-6, relax=True, p_initial=16, p_min=4)

    def run(dl):
        h = FmmBem(v, t, kernel=FMMBEM_STOKES, gauss_k=3, ncrit=150, theta=0.5, p_max=16, precision=FMMBEM_MIXED)
        if dl:
            h.set_device_loop(True)
        b = torch.tensor(np.tile([1.0, 0.0, 0.0], len(t)), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        r = h.solve(b, x, **sk)
        torch.cuda.synchronize()
        out = (r, x.cpu().numpy())
        h.close()
        return out

    (rh, xh), (rd, xd) = run(False), run(True)
    assert rh["converged"] and rd["converged"]
    _orders_follow_rule(rd, sk["tol"], sk["p_initial"], sk["p_min"], True)
    assert abs(rd["iters"] - rh["iters"]) <= 1
    assert rd["true_res"] < 2e-6
    assert _rel(xd, xh) < 1e-4


def test_device_loop_argument_checks(torch_cuda, sphere1280):
    from paper_1506_05957_gb300 import FmmBem, lib
    h = FmmBem(sphere1280["v"], sphere1280["t"], gauss_k=4, ncrit=150, theta=0.5, p_max=8)
    assert lib().fmmbem_set_device_loop(h.h, 2) < 0  # only 0 and 1
    assert lib().fmmbem_set_device_loop(h.h, 1) == 0
    assert lib().fmmbem_set_device_loop(h.h, 0) == 0
    h.close()
