"""Batched Stokes handles (opts.nrhs up to 8, the 8 right-hand sides of the red-blood-cell
configuration of Sec. 3.3): one mat-vec evaluates every vector, one launch per pass, and
fmmbem_solve_batch runs the relaxed GMRES solves in lockstep. Parity against single-vector
handles and against the oracle's Stokeslet operator, through the C ABI.

The geometry is the configuration's at a small size: Evans-Fung cells (eq.
rbc_parameterization) of 512 panels placed by the same seeded recipe, with uniform far-field
velocities U = e_x, e_y, e_z and five seeded unit vectors.

Tolerances: the batch computes the same sums as single-vector handles in another order (FP64:
1e-12; mixed precision: FP32 rounding and the order of the far field's atomic sums, 2e-6);
sampled rows of the p = 16 mixed mat-vec within 1e-5 of the oracle's; solves at tol 1e-5:
the oracle residual of every solution within 2 tol. The first-kind tractions are determined
only up to c n per body (Sec. 2.2 operator's null space), so solutions are compared through
residuals and body forces, not element by element.
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
def cells(torch_cuda):
    from oracle import dense, panels
    from synth import evans_fung_cell, place_cells
    cv, ct = evans_fung_cell(3)  # 512 panels per cell
    v, t, body = place_cells(cv, ct, 3, box=12.0, min_gap=0.5, seed=0)
    _, _, S = panels.geometry(v, t)
    rng = np.random.default_rng(0)
    U = [np.eye(3)[a] for a in range(3)]
    for _ in range(5):
        u = rng.standard_normal(3)
        U.append(u / np.linalg.norm(u))
    mu = 1e-3
    M = dense.Mesh(v, t, k=3)
    A = M.stokes_matrix(mu=mu)
    return dict(v=v, t=t, body=body, S=S, U=np.array(U), mu=mu, M=M, A=A)


def _dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _pair(c, nrhs, **kw):
    from paper_1506_05957_gb300 import FmmBem, FMMBEM_STOKES
    kw.setdefault("ncrit", 60)
    common = dict(kernel=FMMBEM_STOKES, gauss_k=3, theta=0.5, mu=c["mu"], body_of_panel=c["body"])
    single = FmmBem(c["v"], c["t"], **common, **kw)
    batch = FmmBem(c["v"], c["t"], nrhs=nrhs, **common, **kw)
    return single, batch


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stokes_batched_matvec_equals_single(torch_cuda, cells, precision):
    torch = torch_cuda
    from paper_1506_05957_gb300 import FMMBEM_FP64, FMMBEM_MIXED
    c = cells
    prec = FMMBEM_FP64 if precision == "fp64" else FMMBEM_MIXED
    single, batch = _pair(c, 8, precision=prec)
    n = 3 * len(c["t"])
    X = np.random.default_rng(7).standard_normal((8, n))
    xb = _dev(torch, X.reshape(-1))
    yb = torch.zeros_like(xb)
    tol = 1e-12 if precision == "fp64" else 2e-6
    for p in (4, 10, 16):
        batch.matvec(p, xb, yb)
        batch.check_waits()
        Yb = yb.cpu().numpy().reshape(8, n)
        for q in range(8):
            y = torch.zeros(n, dtype=torch.float64, device="cuda")
            single.matvec(p, _dev(torch, X[q]), y)
            assert rel(Yb[q], y.cpu().numpy()) < tol, (p, q, rel(Yb[q], y.cpu().numpy()))
    batch.matvec_direct(xb, yb)
    Yb = yb.cpu().numpy().reshape(8, n)
    for q in range(8):
        assert rel(Yb[q], c["A"] @ X[q]) < (1e-12 if precision == "fp64" else 2e-6), q


def test_stokes_batched_matvec_sampled_oracle_rows(torch_cuda, cells):
    torch = torch_cuda
    c = cells
    _, batch = _pair(c, 5, ncrit=150)  # a batch of another size, at the bench's leaf size
    n = 3 * len(c["t"])
    X = np.random.default_rng(8).standard_normal((5, n))
    xb = _dev(torch, X.reshape(-1))
    yb = torch.zeros_like(xb)
    batch.matvec(16, xb, yb)
    batch.check_waits()
    Yb = yb.cpu().numpy().reshape(5, -1, 3)
    rows = np.sort(np.random.default_rng(9).choice(len(c["t"]), 64, replace=False))
    for q in range(5):
        ref = c["M"].stokes_apply(X[q], mu=c["mu"], rows=rows)
        assert rel(Yb[q][rows], ref) < 1e-5, q


def test_stokes_batched_relaxed_solve(torch_cuda, cells):
    torch = torch_cuda
    from oracle.schedule import schedule
    c = cells
    tol = 1e-5
    single, batch = _pair(c, 8, p_max=16)
    nt = len(c["t"])
    B = np.stack([np.tile(u, nt) for u in c["U"]])
    b = _dev(torch, B.reshape(-1))
    x = torch.zeros_like(b)
    r = batch.solve_batch(b, x, tol=tol, relax=True, p_initial=16, p_min=4)
    assert r["converged"], r
    assert r["p_hist"][0] == 16 and all(4 <= p <= 16 for p in r["p_hist"])
    X = x.cpu().numpy().reshape(8, -1)
    F = np.zeros((8, 3))
    for q in range(8):
        assert rel(c["A"] @ X[q], B[q]) < 2 * tol, q
        assert r["true_res"][q] < 2 * tol
        xs = torch.zeros(3 * nt, dtype=torch.float64, device="cuda")
        rs = single.solve(_dev(torch, B[q]), xs, tol=tol, relax=True, p_initial=16, p_min=4)
        print("system", q, "batched iters", r["iters"][q], "alone", rs["iters"])
        assert abs(r["iters"][q] - rs["iters"]) <= 2
        assert rs["p_hist"] == schedule(tol, rs["res_hist"][:-1], 16, 4)
        # per-cell forces through the batch handle (vector q of the batch)
        Fq = batch.body_integrals(x[q * 3 * nt:(q + 1) * 3 * nt])
        Fs = single.body_integrals(xs)
        assert np.max(np.abs(Fq - Fs)) < 1e-4 * np.max(np.abs(Fs))
        F[q] = Fq.sum(0)
    # every cell's drag opposes its imposed velocity, and the resistance matrix of the three
    # unit motions is symmetric (reciprocal theorem)
    assert np.all(np.einsum("qa,qa->q", F, c["U"]) < 0)
    R = F[:3]
    assert np.max(np.abs(R - R.T)) < 1e-2 * np.max(np.abs(R))
    # the five other velocities are linear combinations of the first three
    for q in range(3, 8):
        assert rel(F[q], c["U"][q] @ R) < 1e-3
