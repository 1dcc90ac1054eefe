"""Refined solves (FMMBEM_MIXED_REFINED): FP64 residuals around the relaxed mixed-precision
GMRES reach tolerances below what the FP32 passes resolve (about 1e-6 relative).

At tol 1e-8 on the 1280-panel sphere with p_initial = 16 (FP64 FMM error below 1e-7):
  - the solve converges with its FP64 true residual <= tol;
  - its solution agrees with the all-FP64 relaxed solve on the same handle to 1e-6
    (both meet ||b - A_16 x|| <= 1e-8 ||b||; the difference is bounded by the conditioning);
  - the dense oracle residual is below 2e-7, under the mixed-precision floor, and within 1e-5
    of the oracle's LU solution, the bar of the other solves.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_refined_solve_reaches_fp64_accuracy():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05957_gb300 import build, FmmBem, FMMBEM_FP64, FMMBEM_MIXED, FMMBEM_MIXED_REFINED
    build.build()
    from oracle import dense, panels
    from synth import icosphere, point_charge_dirichlet
    v, t = icosphere(3)
    M = dense.Mesh(v, t, k=4)
    c, _, _ = panels.geometry(v, t)
    phi = point_charge_dirichlet(c)
    b_ref = 0.5 * phi + M.laplace_apply(phi, kind="dl")
    A = M.laplace_matrix()
    x_lu = np.linalg.solve(A, b_ref)
    h = FmmBem(v, t, gauss_k=4, ncrit=150, theta=0.5, p_max=16, precision=FMMBEM_MIXED_REFINED)
    b = torch.tensor(b_ref, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    r = h.solve(b, x, tol=1e-8, relax=True, p_initial=16, p_min=3)
    print("refined: iters", r["iters"], "true residual", r["true_res"], "p", r["p_hist"])
    assert r["converged"] and r["true_res"] <= 1e-8
    assert abs(r["res_hist"][-1] - r["true_res"]) <= 1e-3 * r["true_res"]
    xr = x.cpu().numpy()
    res = np.linalg.norm(A @ xr - b_ref) / np.linalg.norm(b_ref)
    print("dense oracle residual", res, "error vs LU", np.linalg.norm(xr - x_lu) / np.linalg.norm(x_lu))
    assert res < 2e-7
    assert np.linalg.norm(xr - x_lu) / np.linalg.norm(x_lu) < 1e-5
    h.set_precision(FMMBEM_FP64)
    x64 = torch.zeros_like(b)
    r64 = h.solve(b, x64, tol=1e-8, relax=True, p_initial=16, p_min=3)
    assert r64["converged"]
    assert np.linalg.norm(xr - x64.cpu().numpy()) / np.linalg.norm(x64.cpu().numpy()) < 1e-6
    # plain mixed precision stalls above the refined result's residual at this tolerance
    h.set_precision(FMMBEM_MIXED)
    xm = torch.zeros_like(b)
    rm = h.solve(b, xm, tol=1e-8, relax=True, p_initial=16, p_min=3)
    res_m = np.linalg.norm(A @ xm.cpu().numpy() - b_ref) / np.linalg.norm(b_ref)
    print("mixed at tol 1e-8: converged", rm["converged"], "dense residual", res_m)
    assert res_m > res
    h.close()
