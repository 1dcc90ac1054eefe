"""GPU checks of the boundary options: the near-singular rule's point count (opts.near_k) and
the per-body integrals of a multi-body mesh (mesh.body_of_panel), through the C ABI.

Tolerances: the direct FP64 operators differ from the oracle's only in summation order (1e-12);
body integrals are FP64 sums whose order differs (1e-12 of the largest |S x| sum).
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("near_k", [6, 12, 30, 42])
def test_near_rule_point_count(torch_cuda, near_k):
    torch = torch_cuda
    from oracle import dense
    from paper_1506_05957_gb300 import FmmBem, FMMBEM_FP64, FMMBEM_LAPLACE, FMMBEM_STOKES
    from synth import icosphere
    v, t = icosphere(3)
    x = np.random.default_rng(3).standard_normal(len(t))
    ref = dense.Mesh(v, t, k=4, near_k=near_k).laplace_apply(x)
    h = FmmBem(v, t, kernel=FMMBEM_LAPLACE, gauss_k=4, ncrit=150, theta=0.5, precision=FMMBEM_FP64, near_k=near_k)
    y = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    h.matvec_direct(torch.tensor(x, device="cuda"), y)
    assert rel(y.cpu().numpy(), ref) < 1e-12
    # the rule changes the near entries: the default's operator differs
    ref20 = dense.Mesh(v, t, k=4).laplace_apply(x)
    assert rel(ref, ref20) > 1e-9
    h.close()
    v2, t2 = icosphere(2)
    u = np.random.default_rng(4).standard_normal((len(t2), 3))
    refs = dense.Mesh(v2, t2, k=3, near_k=near_k).stokes_apply(u, mu=1.0)
    hs = FmmBem(v2, t2, kernel=FMMBEM_STOKES, gauss_k=3, ncrit=60, theta=0.5, precision=FMMBEM_FP64, near_k=near_k)
    ys = torch.zeros(hs.n, dtype=torch.float64, device="cuda")
    hs.matvec_direct(torch.tensor(u.reshape(-1), device="cuda"), ys)
    assert rel(ys.cpu().numpy().reshape(-1, 3), refs) < 1e-12
    hs.close()


def test_body_integrals_two_bodies(torch_cuda):
    torch = torch_cuda
    from oracle import panels
    from paper_1506_05957_gb300 import FmmBem, FMMBEM_LAPLACE, FMMBEM_STOKES
    from synth import icosphere, ellipsoid
    v1, t1 = icosphere(3, radius=1.0, center=(-2.0, 0.0, 0.0))
    v2, t2 = ellipsoid(2, axes=(0.5, 1.0, 1.5), center=(2.0, 0.5, 0.0))
    v = np.vstack([v1, v2])
    t = np.vstack([t1, t2 + len(v1)])
    body = np.concatenate([np.zeros(len(t1), np.int32), np.ones(len(t2), np.int32)])
    _, _, S = panels.geometry(v, t)
    rng = np.random.default_rng(5)
    for kernel, dof, k in ((FMMBEM_LAPLACE, 1, 4), (FMMBEM_STOKES, 3, 3)):
        h = FmmBem(v, t, kernel=kernel, gauss_k=k, ncrit=100, theta=0.5, body_of_panel=body)
        assert h.n_bodies == 2
        x = rng.standard_normal((len(t), dof))
        got = h.body_integrals(torch.tensor(x.reshape(-1), device="cuda"))
        want = np.array([(S[body == b, None] * x[body == b]).sum(0) for b in range(2)])
        assert got.shape == (2, dof)
        assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(S[:, None] * x)) * len(t)
        h.close()
    # one body when the mesh names none
    h = FmmBem(v, t, kernel=FMMBEM_LAPLACE, gauss_k=4, ncrit=100, theta=0.5)
    x = rng.standard_normal(len(t))
    got = h.body_integrals(torch.tensor(x, device="cuda"))
    assert got.shape == (1, 1) and abs(got[0, 0] - np.sum(S * x)) < 1e-12 * np.sum(np.abs(S * x))
    h.close()
