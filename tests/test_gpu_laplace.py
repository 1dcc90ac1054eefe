"""GPU parity of the Laplace path against the oracle, through the C ABI.

Tolerances (written per test) follow from the arithmetic:
  - direct FP64 operator vs oracle: same quadrature, only summation order differs -> 1e-12;
  - FMM in FP64: truncation error falling with p; at p = 16 and theta = 0.5 below 1e-7;
  - mixed precision (FP32 passes, FP64 tile sums and corrections): below 1e-5 at p >= 8;
  - solves at tol 1e-6: oracle residual of the GPU solution <= 2 tol (robust to the
    condition number), solution error vs the oracle's LU solution <= 1e-5 relative.
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
    A = M.laplace_matrix()
    return dict(v=v, t=t, M=M, phi=phi, b=b, A=A, x_lu=np.linalg.solve(A, b))


def _h(torch, v, t, **kw):
    from paper_1506_05957_gb300 import FmmBem
    kw.setdefault("gauss_k", 4)
    kw.setdefault("ncrit", 150)
    kw.setdefault("theta", 0.5)
    return FmmBem(v, t, **kw)


def _dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_direct_operator_matches_oracle(torch_cuda, sphere1280):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64, FMMBEM_MIXED
    s = sphere1280
    x = np.random.default_rng(0).standard_normal(len(s["t"]))
    ref = s["A"] @ x
    h = _h(torch, s["v"], s["t"], precision=FMMBEM_FP64)
    y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.matvec_direct(_dev(torch, x), y)
    assert rel(y.cpu().numpy(), ref) < 1e-12
    h.set_precision(FMMBEM_MIXED)
    h.matvec_direct(_dev(torch, x), y)
    assert rel(y.cpu().numpy(), ref) < 2e-6


def test_rhs_matches_oracle(torch_cuda, sphere1280):
    torch = torch_cuda
    s = sphere1280
    h = _h(torch, s["v"], s["t"])
    b = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.rhs(_dev(torch, s["phi"]), b)
    assert rel(b.cpu().numpy(), s["b"]) < 1e-12


@pytest.mark.parametrize("ncrit", [40, 150, 600])
def test_fmm_fp64_error_falls_with_p(torch_cuda, sphere1280, ncrit):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64
    s = sphere1280
    x = np.random.default_rng(1).standard_normal(len(s["t"]))
    ref = s["A"] @ x
    h = _h(torch, s["v"], s["t"], ncrit=ncrit, precision=FMMBEM_FP64)
    xd = _dev(torch, x)
    y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    errs = []
    for p in (1, 2, 4, 6, 8, 10, 12, 16):
        h.matvec(p, xd, y)
        errs.append(rel(y.cpu().numpy(), ref))
    print("ncrit", ncrit, "errors by p", ["%.2e" % e for e in errs], h.stats())
    for a, b in zip(errs, errs[1:]):
        assert b < a * 1.05 or b < 1e-13
    # truncation error of a theta = 0.5 expansion: ~ 2^-(p+1) or better
    for p, e in zip((1, 2, 4, 6, 8, 10, 12, 16), errs):
        assert e < 2.0 ** -(p + 1)
    assert errs[-1] < 1e-7


def test_fmm_mixed_precision_close_to_oracle(torch_cuda, sphere1280):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_MIXED
    s = sphere1280
    x = np.random.default_rng(2).standard_normal(len(s["t"]))
    ref = s["A"] @ x
    h = _h(torch, s["v"], s["t"], precision=FMMBEM_MIXED)
    y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    errs = {}
    for p in (4, 8, 12, 16):
        h.matvec(p, _dev(torch, x), y)
        errs[p] = rel(y.cpu().numpy(), ref)
    print("mixed errors", errs)
    assert errs[12] < 1e-5 and errs[16] < 1e-5


def test_relaxed_solve_matches_oracle(torch_cuda, sphere1280):
    torch = torch_cuda
    from oracle.gmres import gmres
    from oracle.schedule import schedule
    s = sphere1280
    tol = 1e-6
    h = _h(torch, s["v"], s["t"], p_max=12)
    b = _dev(torch, s["b"])
    x = torch.zeros_like(b)
    r = h.solve(b, x, tol=tol, relax=True, p_initial=10, p_min=3)
    assert r["converged"]
    xs = x.cpu().numpy()
    # the p schedule is exactly the relaxation rule applied to the residuals the solve saw
    assert r["p_hist"] == schedule(tol, r["res_hist"][:-1], 10, 3)
    assert r["p_hist"][0] == 10 and min(r["p_hist"]) < 10
    res = rel(s["A"] @ xs, s["b"])
    assert res < 2 * tol
    assert rel(xs, s["x_lu"]) < 1e-5
    # iteration counts: relaxed ~ fixed ~ exact GMRES (the paper's observation, Sec. 3.1). The GPU
    # iterates on the mixed-precision FMM operator at p <= 10, which differs from the dense matrix by
    # ~1e-6 relative, so the residual estimate may cross tol one step earlier or later than exact
    # GMRES does (observed: 16 relaxed, 16 fixed, 15 exact); one step is the allowance.
    x2 = torch.zeros_like(b)
    r2 = h.solve(b, x2, tol=tol, relax=False, p_initial=10, p_min=3)
    _, it_oracle, _ = gmres(lambda u, k: s["A"] @ u, s["b"], tol=tol, restart=50, max_iter=100)
    print("iters relaxed/fixed/oracle", r["iters"], r2["iters"], it_oracle, r["p_hist"])
    assert abs(r["iters"] - r2["iters"]) <= 1
    assert abs(r2["iters"] - it_oracle) <= 1
    assert all(p == 10 for p in r2["p_hist"])


def test_fp64_fixed_p_solve(torch_cuda, sphere1280):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64
    s = sphere1280
    h = _h(torch, s["v"], s["t"], p_max=16, precision=FMMBEM_FP64)
    b = _dev(torch, s["b"])
    x = torch.zeros_like(b)
    r = h.solve(b, x, tol=1e-10, relax=False, p_initial=16, p_min=16)
    assert r["converged"]
    assert rel(x.cpu().numpy(), s["x_lu"]) < 1e-6
    assert r["true_res"] < 1e-7


def test_solve_host_buffers(torch_cuda, sphere1280):
    torch = torch_cuda
    s = sphere1280
    h = _h(torch, s["v"], s["t"], p_max=12)
    b = np.ascontiguousarray(s["b"])
    x = np.zeros_like(b)
    r = h.solve_host(b, x, tol=1e-6, relax=True, p_initial=10, p_min=3)
    xd = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    r2 = h.solve(_dev(torch, b), xd, tol=1e-6, relax=True, p_initial=10, p_min=3)
    # the M2L scatter uses atomic additions, so two solves differ by rounding only:
    # same iteration count, solutions within the solver tolerance of each other
    assert abs(r["iters"] - r2["iters"]) <= 1
    assert rel(x, xd.cpu().numpy()) < 1e-6


def test_tiny_and_degenerate_trees(torch_cuda):
    """20 panels (no far field at all), one leaf holding everything, and p = 1."""
    torch = torch_cuda
    from oracle import dense
    from synth import icosphere
    from paper_1506_05957_gb300 import FMMBEM_FP64
    for lev, ncrit in ((0, 4), (1, 10000), (2, 4)):
        v, t = icosphere(lev)
        M = dense.Mesh(v, t, k=4)
        x = np.random.default_rng(lev).standard_normal(len(t))
        ref = M.laplace_apply(x)
        h = _h(torch, v, t, ncrit=ncrit, precision=FMMBEM_FP64)
        y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
        h.matvec(16, _dev(torch, x), y)
        assert rel(y.cpu().numpy(), ref) < 1e-7, (lev, ncrit)
        h.matvec(1, _dev(torch, x), y)
        assert rel(y.cpu().numpy(), ref) < 0.3


def test_invalid_arguments_are_errors(torch_cuda, sphere1280):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FmmBemError
    s = sphere1280
    h = _h(torch, s["v"], s["t"], p_max=8)
    x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    for p in (0, 9, 17):
        with pytest.raises(FmmBemError):
            h.matvec(p, x, y)
    with pytest.raises(FmmBemError):
        h.matvec(4, x, x)
    with pytest.raises(FmmBemError):
        h.stokes_dl_apply(x, y)
    with pytest.raises(FmmBemError):
        h.solve(x, y, tol=1e-6, p_initial=8, p_min=9)
    # zero right-hand side: zero solution, no iterations
    r = h.solve(x, y, tol=1e-6, p_initial=8, p_min=3)
    assert r["iters"] == 0 and float(y.abs().max()) == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_m2l_formulations_agree(torch_cuda, sphere1280, precision):
    """Operator-table GEMM (SIMT), on-the-fly gather and, in mixed precision, the
    tcgen05 3xTF32 path compute the same M2L sums."""
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64, FMMBEM_MIXED
    from paper_1506_05957_gb300.binding import FMMBEM_M2L_GATHER, FMMBEM_M2L_TABLES, FMMBEM_M2L_TENSOR
    s = sphere1280
    h = _h(torch, s["v"], s["t"], ncrit=40, precision=FMMBEM_FP64 if precision == "fp64" else FMMBEM_MIXED)
    x = _dev(torch, np.random.default_rng(5).standard_normal(h.n))
    modes = [FMMBEM_M2L_TABLES, FMMBEM_M2L_GATHER] + ([FMMBEM_M2L_TENSOR] if precision == "mixed" else [])
    tol = 1e-13 if precision == "fp64" else 2e-6
    for p in (1, 3, 7, 12, 15, 16):
        ys = []
        for mode in modes:
            h.set_m2l_mode(mode)
            y = torch.zeros_like(x)
            h.matvec(p, x, y)
            ys.append(y.cpu().numpy())
        for y in ys[1:]:
            assert rel(y, ys[0]) < tol, p


@pytest.mark.parametrize("ncrit", [40, 150, 600])
def test_p2p_variants_agree(torch_cuda, sphere1280, ncrit):
    """The four near-field schedules compute the same FP32 sums (summation order differs):
    shared tiles, sliced L1, bulk-copied stages and source lanes. ncrit 600 puts up to
    150 targets in a leaf (several target passes), ncrit 40 gives leaves with more P2P
    pairs than one shared-memory chunk of records holds."""
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_MIXED
    s = sphere1280
    h = _h(torch, s["v"], s["t"], ncrit=ncrit, precision=FMMBEM_MIXED)
    x = _dev(torch, np.random.default_rng(9).standard_normal(h.n))
    ref = s["A"] @ x.cpu().numpy()
    ys = []
    for variant in (0, 1, 2, 3):
        h.set_p2p_variant(variant)
        y = torch.zeros_like(x)
        h.matvec(16, x, y)
        ys.append(y.cpu().numpy())
    for v, y in enumerate(ys):
        assert rel(y, ys[0]) < 2e-6, v
        assert rel(y, ref) < 1e-5, v
    with pytest.raises(Exception):
        h.set_p2p_variant(4)



def test_autotune_keeps_results(torch_cuda, sphere1280):
    """The autotuner only chooses among schedules of the same sums (the near-field schedule, and
    tensor-core or SIMT translations per order p): the solve after tuning matches the oracle as
    before, and every choice is one of the offered ones."""
    torch = torch_cuda
    s = sphere1280
    h = _h(torch, s["v"], s["t"], p_max=12)
    ch = h.autotune(3, 12)
    print("autotune choices", ch)
    assert set(ch) == {0} | set(range(3, 13)) and ch[0] in (0, 1, 2, 3)
    assert all(ch[p] in (0, 1, 2, 3) for p in range(3, 13))
    b = _dev(torch, s["b"])
    x = torch.zeros_like(b)
    r = h.solve(b, x, tol=1e-6, relax=True, p_initial=10, p_min=3)
    assert r["converged"]
    assert rel(x.cpu().numpy(), s["x_lu"]) < 1e-5
    with pytest.raises(Exception):
        h.autotune(0, 5)


def test_tuned_create_picks_a_candidate_leaf_capacity(torch_cuda, sphere1280):
    """fmmbem_create_tuned builds the tree at each candidate leaf capacity and keeps the one
    whose mat-vecs over [p_lo, p_hi] are fastest; the kept handle solves like any other."""
    torch = torch_cuda
    from paper_1506_05957_gb300 import FmmBem
    s = sphere1280
    h = FmmBem.tuned(s["v"], s["t"], ncrit_candidates=(40, 80, 150), p_lo=3, p_hi=10, gauss_k=4, theta=0.5,
                     p_max=12)
    print("tuned ncrit", h.tuned_ncrit, "summed mat-vec ms", h.tuned_ms)
    assert h.tuned_ncrit in (40, 80, 150) and h.tuned_ms > 0.0
    b = _dev(torch, s["b"])
    x = torch.zeros_like(b)
    r = h.solve(b, x, tol=1e-6, relax=True, p_initial=10, p_min=3)
    assert r["converged"] and rel(x.cpu().numpy(), s["x_lu"]) < 1e-5
    h.close()
