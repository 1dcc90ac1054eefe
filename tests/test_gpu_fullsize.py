"""Parity at the benchmark's full size (81920 panels, icosahedron refined 6 times), in
the launch configuration bench.py times (K = 4, theta = 0.5, ncrit = 150, p_max = 16,
mixed precision, tensor-core M2L, bulk-copy P2P): outputs the oracle can compute row by
row are sampled and compared element by element, through the C ABI."""
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
def big(torch_cuda):
    from oracle import dense, panels
    from synth import icosphere, point_charge_dirichlet
    v, t = icosphere(6)
    c, _, _ = panels.geometry(v, t)
    return dict(v=v, t=t, M=dense.Mesh(v, t, k=4), phi=point_charge_dirichlet(c),
                rows=np.sort(np.random.default_rng(3).choice(len(t), 512, replace=False)))


def _h(v, t, **kw):
    from paper_1506_05957_gb300 import FmmBem, FMMBEM_MIXED
    return FmmBem(v, t, gauss_k=4, ncrit=150, theta=0.5, p_max=16, precision=FMMBEM_MIXED, **kw)


def test_fullsize_matvec_sampled_rows(torch_cuda, big):
    torch = torch_cuda
    h = _h(big["v"], big["t"])
    x = np.random.default_rng(4).standard_normal(h.n)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(xd)
    ref = big["M"].laplace_apply(x, rows=big["rows"])
    scale = np.sqrt(np.mean(ref * ref))
    for p, tol in ((12, 1e-5), (16, 1e-5), (6, 2e-3), (3, 3e-2)):
        h.matvec(p, xd, y)
        got = y.cpu().numpy()[big["rows"]]
        err = np.abs(got - ref)
        print("p", p, "max abs err / rms", err.max() / scale, "rel L2", np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
        assert err.max() < 5 * tol * scale


def test_fullsize_rhs_sampled_rows(torch_cuda, big):
    torch = torch_cuda
    h = _h(big["v"], big["t"])
    b = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.rhs(torch.tensor(big["phi"], dtype=torch.float64, device="cuda"), b)
    ref = 0.5 * big["phi"][big["rows"]] + big["M"].laplace_apply(big["phi"], kind="dl", rows=big["rows"])
    got = b.cpu().numpy()[big["rows"]]
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_fullsize_relaxed_solve_sampled_residual(torch_cuda, big):
    torch = torch_cuda
    from oracle.schedule import schedule
    h = _h(big["v"], big["t"])
    phi = torch.tensor(big["phi"], dtype=torch.float64, device="cuda")
    b = torch.zeros_like(phi)
    h.rhs(phi, b)
    x = torch.zeros_like(b)
    r = h.solve(b, x, tol=1e-6, relax=True, p_initial=12, p_min=3)
    assert r["converged"] and r["true_res"] < 2e-6
    assert r["p_hist"] == schedule(1e-6, r["res_hist"][:-1], 12, 3)
    rows = big["rows"]
    bs = b.cpu().numpy()[rows]
    res = big["M"].laplace_apply(x.cpu().numpy(), rows=rows) - bs
    print("iters", r["iters"], "sampled oracle residual", np.linalg.norm(res) / np.linalg.norm(bs))
    assert np.linalg.norm(res) / np.linalg.norm(bs) < 2e-6
