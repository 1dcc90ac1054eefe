"""GPU parity of the Stokes path (Stokeslet single layer, four-Laplace far field,
stresslet double layer) against the oracle, through the C ABI.
Tolerances as in test_gpu_laplace; the drag is checked against 6 pi mu a U."""
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
def sphere(torch_cuda):
    from oracle import dense, panels
    from synth import icosphere
    v, t = icosphere(3)
    M = dense.Mesh(v, t, k=3)
    _, n, S = panels.geometry(v, t)
    A = M.stokes_matrix(mu=1.0)
    return dict(v=v, t=t, M=M, A=A, n=n, S=S)


def _h(v, t, **kw):
    from paper_1506_05957_gb300 import FmmBem, FMMBEM_STOKES
    kw.setdefault("gauss_k", 3)
    kw.setdefault("ncrit", 150)
    kw.setdefault("theta", 0.5)
    return FmmBem(v, t, kernel=FMMBEM_STOKES, **kw)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_stokes_direct_matches_oracle(torch_cuda, sphere):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64
    s = sphere
    x = np.random.default_rng(0).standard_normal(3 * len(s["t"]))
    h = _h(s["v"], s["t"], precision=FMMBEM_FP64)
    y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.matvec_direct(torch.tensor(x, device="cuda"), y)
    assert rel(y.cpu().numpy(), s["A"] @ x) < 1e-12


def test_stresslet_matches_oracle(torch_cuda, sphere):
    torch = torch_cuda
    s = sphere
    u = np.random.default_rng(1).standard_normal(3 * len(s["t"]))
    h = _h(s["v"], s["t"])
    y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.stokes_dl_apply(torch.tensor(u, device="cuda"), y)
    ref = s["M"].stokes_apply(u, kind="dl").reshape(-1)
    assert rel(y.cpu().numpy(), ref) < 1e-12


def test_stokes_fmm_error_falls_with_p(torch_cuda, sphere):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64, FMMBEM_MIXED
    s = sphere
    x = np.random.default_rng(2).standard_normal(3 * len(s["t"]))
    ref = s["A"] @ x
    h = _h(s["v"], s["t"], precision=FMMBEM_FP64)
    y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    xd = torch.tensor(x, device="cuda")
    errs = []
    for p in (1, 2, 4, 8, 12, 16):
        h.matvec(p, xd, y)
        errs.append(rel(y.cpu().numpy(), ref))
    print("stokes fp64 errors", ["%.2e" % e for e in errs])
    for a, b in zip(errs, errs[1:]):
        assert b < a * 1.05
    assert errs[-1] < 1e-7
    h.set_precision(FMMBEM_MIXED)
    h.matvec(16, xd, y)
    e = rel(y.cpu().numpy(), ref)
    print("stokes mixed p16", e)
    assert e < 1e-5


def test_stokes_relaxed_solve_drag(torch_cuda, sphere):
    torch = torch_cuda
    from oracle.schedule import schedule
    s = sphere
    tol = 1e-5
    h = _h(s["v"], s["t"], p_max=16)
    U = np.tile([1.0, 0.0, 0.0], len(s["t"]))
    b = torch.tensor(U, device="cuda")
    x = torch.zeros_like(b)
    r = h.solve(b, x, tol=tol, relax=True, p_initial=16, p_min=4)
    assert r["converged"]
    assert r["p_hist"] == schedule(tol, r["res_hist"][:-1], 16, 4)
    tr = x.cpu().numpy().reshape(-1, 3)
    F = float(np.sum(tr[:, 0] * s["S"]))
    print("drag", F, "iters", r["iters"], r["p_hist"])
    assert abs(F / (-6.0 * np.pi) - 1.0) < 1e-2
    assert rel(s["A"] @ tr.reshape(-1), U) < 2 * tol
    x2 = torch.zeros_like(b)
    r2 = h.solve(b, x2, tol=tol, relax=False, p_initial=16, p_min=4)
    assert abs(r["iters"] - r2["iters"]) <= 2


def test_cell_cluster_high_order_stays_finite():
    """Clusters of red-blood-cell surfaces in a large box leave coarse cells that hold a small
    piece of surface: with the cluster radii alone such a cell could be accepted for M2L with a
    centre offset much smaller than its side, and the FP32 translation operators of degree up
    to 2p = 32 overflowed (NaN mat-vecs at p = 16 on these two placements). The acceptance
    criterion also asks for centres at least the larger side apart: the p = 16 mat-vecs are
    finite and match the oracle's Stokeslet rows, and the relaxed solves converge."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05957_gb300 import build, FmmBem, FMMBEM_MIXED, FMMBEM_STOKES
    build.build()
    from oracle import dense
    from synth import evans_fung_cell, place_cells
    cv, ct = evans_fung_cell(4)
    for n_cells, seed in ((4, 1016323256), (16, 995813860)):
        v, t, _ = place_cells(cv, ct, n_cells, box=40.0, min_gap=0.5, seed=seed)
        h = FmmBem(v, t, kernel=FMMBEM_STOKES, gauss_k=3, ncrit=150, theta=0.5, p_max=16, precision=FMMBEM_MIXED)
        x = np.random.default_rng(seed % 1000).standard_normal(h.n)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(xd)
        h.matvec(16, xd, y)
        h.check_waits()
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        rows = np.sort(np.random.default_rng(3).choice(len(t), 48, replace=False))
        ref = dense.Mesh(v, t, k=3).stokes_apply(x, rows=rows).reshape(-1)
        g = got.reshape(-1, 3)[rows].reshape(-1)
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-5
        b = torch.tensor(np.tile([1.0, 0.0, 0.0], len(t)), dtype=torch.float64, device="cuda")
        sol = torch.zeros_like(b)
        r = h.solve(b, sol, tol=1e-6, relax=True, p_initial=16, p_min=4)
        assert r["converged"] and np.isfinite(r["true_res"]) and r["true_res"] < 2e-6
        h.close()
