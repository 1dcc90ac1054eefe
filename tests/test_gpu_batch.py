"""Batched Laplace handles (opts.nrhs = 4): one mat-vec evaluates four vectors, and
fmmbem_solve_batch runs four relaxed GMRES solves in lockstep. Parity against single-vector
handles and against the oracle, through the C ABI.

Tolerances: the batched mat-vec computes the same sums as four single ones in another
order (FP64: 1e-12; mixed precision: FP32 rounding of the packed strengths and the M2L
atomics, 2e-6). Batched solves: each solution within 1e-5 of the oracle's LU solution (the
single-vector solve's bar), the oracle residual within 2 tol.
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
    from synth import icosphere
    v, t = icosphere(3)
    M = dense.Mesh(v, t, k=4)
    c, _, _ = panels.geometry(v, t)
    A = M.laplace_matrix()
    rhs = []
    for z0 in ((0.0, 0.0, 3.0), (2.5, 0.5, 0.0), (-0.3, -2.2, 1.1)):
        d = c - np.asarray(z0)
        phi = 1.0 / (4.0 * np.pi * np.sqrt((d * d).sum(1)))
        rhs.append(0.5 * phi + M.laplace_apply(phi, kind="dl"))
    rhs.append(np.random.default_rng(3).standard_normal(len(t)))
    return dict(v=v, t=t, A=A, rhs=rhs)


def _dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _pair(v, t, **kw):
    from paper_1506_05957_gb300 import FmmBem
    kw.setdefault("ncrit", 60)
    single = FmmBem(v, t, gauss_k=4, theta=0.5, **kw)
    batch = FmmBem(v, t, gauss_k=4, theta=0.5, nrhs=4, **kw)
    return single, batch


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_matvec_equals_single(torch_cuda, sphere1280, precision):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64, FMMBEM_MIXED
    s = sphere1280
    prec = FMMBEM_FP64 if precision == "fp64" else FMMBEM_MIXED
    single, batch = _pair(s["v"], s["t"], precision=prec)
    n = len(s["t"])
    X = np.random.default_rng(7).standard_normal((4, n))
    xb = _dev(torch, X.reshape(-1))
    yb = torch.zeros_like(xb)
    tol = 1e-12 if precision == "fp64" else 2e-6
    for p in (3, 8, 12):
        batch.matvec(p, xb, yb)
        Yb = yb.cpu().numpy().reshape(4, n)
        for q in range(4):
            y = torch.zeros(n, dtype=torch.float64, device="cuda")
            single.matvec(p, _dev(torch, X[q]), y)
            assert rel(Yb[q], y.cpu().numpy()) < tol, (p, q)
    # the dense operator of the batch handle, vector by vector, against the oracle
    batch.matvec_direct(xb, yb)
    Yb = yb.cpu().numpy().reshape(4, n)
    for q in range(4):
        assert rel(Yb[q], s["A"] @ X[q]) < (1e-12 if precision == "fp64" else 2e-6)


def test_batched_relaxed_solve_matches_oracle(torch_cuda, sphere1280):
    torch = torch_cuda
    s = sphere1280
    tol = 1e-6
    single, batch = _pair(s["v"], s["t"], p_max=12)
    n = len(s["t"])
    B = np.stack(s["rhs"])
    b = _dev(torch, B.reshape(-1))
    x = torch.zeros_like(b)
    r = batch.solve_batch(b, x, tol=tol, relax=True, p_initial=10, p_min=3)
    assert r["converged"], r
    X = x.cpu().numpy().reshape(4, n)
    for q in range(4):
        x_lu = np.linalg.solve(s["A"], B[q])
        assert rel(s["A"] @ X[q], B[q]) < 2 * tol, q
        assert rel(X[q], x_lu) < 1e-5, q
        assert r["true_res"][q] < 2 * tol
        # the same system alone: iteration counts agree (the batch runs each at least as
        # accurately as its own schedule asks)
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        rs = single.solve(_dev(torch, B[q]), xs, tol=tol, relax=True, p_initial=10, p_min=3)
        print("system", q, "batched iters", r["iters"][q], "alone", rs["iters"])
        assert abs(r["iters"][q] - rs["iters"]) <= 2
    # the shared order is the largest any active system asked for: never below p_min
    assert all(3 <= p <= 10 for p in r["p_hist"]) and r["p_hist"][0] == 10


def test_batch_with_zero_and_repeated_systems(torch_cuda, sphere1280):
    torch = torch_cuda
    s = sphere1280
    _, batch = _pair(s["v"], s["t"], p_max=12)
    n = len(s["t"])
    B = np.stack([s["rhs"][0], np.zeros(n), s["rhs"][0], s["rhs"][1]])
    b = _dev(torch, B.reshape(-1))
    x = torch.zeros_like(b)
    r = batch.solve_batch(b, x, tol=1e-6, relax=True, p_initial=10, p_min=3)
    X = x.cpu().numpy().reshape(4, n)
    assert r["iters"][1] == 0 and np.all(X[1] == 0.0)
    # identical systems: equal up to the rounding order of the far field's atomic sums
    assert rel(X[2], X[0]) < 1e-6 and abs(r["iters"][0] - r["iters"][2]) <= 1


def test_batch_argument_errors(torch_cuda, sphere1280):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FmmBem, FmmBemError, FMMBEM_STOKES, FMMBEM_LAYER_DOUBLE
    s = sphere1280
    single, batch = _pair(s["v"], s["t"], p_max=8)
    n = len(s["t"])
    b4 = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    b1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(FmmBemError):
        batch.solve(b4, torch.zeros_like(b4))  # single-system entry on a batched handle
    with pytest.raises(FmmBemError):
        single.solve_batch(b1, torch.zeros_like(b1))
    with pytest.raises(FmmBemError):
        batch.set_layer(FMMBEM_LAYER_DOUBLE)
    with pytest.raises(FmmBemError):
        FmmBem(s["v"], s["t"], kernel=FMMBEM_STOKES, gauss_k=3, nrhs=9)  # beyond FMMBEM_STOKES_BATCH_MAX
    with pytest.raises(FmmBemError):
        FmmBem(s["v"], s["t"], nrhs=3)  # a Laplace batch holds FMMBEM_BATCH vectors
