"""Single multipole/local expansions on the GPU (FP64) against the truncation
bound of eq. multipole_error and its local-expansion counterpart, with the
exact potentials from the oracle's direct sums."""
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


def _ball(rng, n, radius):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * (radius * rng.random(n) ** (1 / 3))[:, None]


@pytest.mark.parametrize("ratio", [1.5, 2.0, 4.0])
def test_multipole_error_bound(torch_cuda, ratio):
    torch = torch_cuda
    from oracle.dense import nbody_laplace
    from paper_1506_05957_gb300 import fmmbem_expansion_eval
    rng = np.random.default_rng(int(ratio * 10))
    a = 0.3
    c = np.array([0.1, -0.2, 0.05])
    src = c + _ball(rng, 200, a)
    q = rng.standard_normal(200)
    dirs = rng.standard_normal((64, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    r = ratio * a
    tgt = c + r * dirs
    exact = nbody_laplace(tgt, src, q)
    s_dev = torch.tensor(np.column_stack([src, q]), dtype=torch.float64, device="cuda")
    t_dev = torch.tensor(tgt, dtype=torch.float64, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    prev = np.inf
    for p in range(0, 17):
        fmmbem_expansion_eval(0, p, c, 0.7, s_dev, t_dev, out)
        err = np.abs(out.cpu().numpy() - exact).max()
        bound = np.abs(q).sum() / (r - a) * (a / r) ** (p + 1)
        assert err <= bound * (1 + 1e-9) + 1e-13, (p, err, bound)
        if p >= 2:
            assert err < prev * 1.5
        prev = err


def test_local_error_bound(torch_cuda):
    torch = torch_cuda
    from oracle.dense import nbody_laplace
    from paper_1506_05957_gb300 import fmmbem_expansion_eval
    rng = np.random.default_rng(5)
    c = np.zeros(3)
    dirs = rng.standard_normal((150, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    rho = 1.0 + rng.random(150)
    src = dirs * rho[:, None]
    q = rng.standard_normal(150)
    r = 0.45
    tgt = _ball(rng, 64, r)
    exact = nbody_laplace(tgt, src, q)
    s_dev = torch.tensor(np.column_stack([src, q]), dtype=torch.float64, device="cuda")
    t_dev = torch.tensor(tgt, dtype=torch.float64, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    rmax = np.linalg.norm(tgt, axis=1).max()
    for p in range(0, 17):
        fmmbem_expansion_eval(1, p, c, 1.3, s_dev, t_dev, out)
        err = np.abs(out.cpu().numpy() - exact).max()
        bound = np.abs(q).sum() / (rho.min() - rmax) * (rmax / rho.min()) ** (p + 1)
        assert err <= bound * (1 + 1e-9) + 1e-13, (p, err, bound)
