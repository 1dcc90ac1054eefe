"""Bounded device waits: a grid-barrier wait of the Arnoldi step that runs out (a poll limit of
a few iterations, so the other blocks cannot have arrived yet) must end the solve with
FMMBEM_ETIMEOUT instead of holding the GPU, reset its state, and leave the handle usable: the
next solve on it matches the oracle. Mat-vecs report their waits through fmmbem_check_waits.

No GPU fault is involved: the barrier's wait is a plain polling loop with no asynchronous
copies or tensor memory in flight, so giving up early only makes the step's results invalid.
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


def test_grid_barrier_timeout_then_normal_solve(torch_cuda):
    torch = torch_cuda
    from oracle import dense, panels, schedule
    from paper_1506_05957_gb300 import FmmBem, FmmBemError, FMMBEM_MIXED
    from paper_1506_05957_gb300.binding import FMMBEM_ETIMEOUT
    from synth import icosphere, point_charge_dirichlet
    v, t = icosphere(3)
    M = dense.Mesh(v, t, k=4)
    c, _, _ = panels.geometry(v, t)
    phi = point_charge_dirichlet(c)
    b_ref = 0.5 * phi + M.laplace_apply(phi, kind="dl")
    h = FmmBem(v, t, gauss_k=4, ncrit=150, theta=0.5, p_max=12, precision=FMMBEM_MIXED)
    b = torch.tensor(b_ref, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    h.set_wait_limit(1)
    with pytest.raises(FmmBemError) as ei:
        h.solve(b, x, tol=1e-6, relax=True, p_initial=10, p_min=3)
    assert ei.value.code == FMMBEM_ETIMEOUT
    h.check_waits()  # the solve cleared what it reported
    h.set_wait_limit(0)
    r = h.solve(b, x, tol=1e-6, relax=True, p_initial=10, p_min=3)
    assert r["converged"]
    assert r["p_hist"] == schedule.schedule(1e-6, r["res_hist"][:-1], 10, 3)
    res = np.linalg.norm(M.laplace_apply(x.cpu().numpy()) - b_ref) / np.linalg.norm(b_ref)
    assert res < 2e-6, res
    # mat-vecs queue asynchronously; their waits are read by fmmbem_check_waits
    y = torch.empty_like(b)
    for p in (3, 12):
        h.matvec(p, x, y)
    h.check_waits()
    h.close()


def test_peak_rates_are_plausible(torch_cuda):
    torch = torch_cuda
    from paper_1506_05957_gb300.binding import (fmmbem_peak, FMMBEM_PEAK_FFMA, FMMBEM_PEAK_FFMA2,
                                                FMMBEM_PEAK_RSQRT, FMMBEM_PEAK_DFMA, FMMBEM_PEAK_TF32)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.07e9 * 1.05  # no rate may exceed what the units could do at the maximum clock (5% margin)
    rate = {}
    for kind, it in ((FMMBEM_PEAK_FFMA, 100000), (FMMBEM_PEAK_FFMA2, 50000), (FMMBEM_PEAK_RSQRT, 20000),
                     (FMMBEM_PEAK_DFMA, 2000), (FMMBEM_PEAK_TF32, 10000)):
        ops, ms = fmmbem_peak(kind, it)
        assert ops > 0 and ms > 0
        rate[kind] = ops / (ms * 1e-3)
    assert 0.2 * sms * 256 * clk < rate[FMMBEM_PEAK_FFMA] < sms * 256 * clk  # 128 FP32 lanes, 2 flop
    assert rate[FMMBEM_PEAK_FFMA2] > 0.9 * rate[FMMBEM_PEAK_FFMA]
    assert rate[FMMBEM_PEAK_RSQRT] < sms * 32 * clk
    assert rate[FMMBEM_PEAK_DFMA] < 0.1 * rate[FMMBEM_PEAK_FFMA]  # FP64 is a small fraction of FP32 here
    assert 0.2e15 < rate[FMMBEM_PEAK_TF32] < 1.5e15  # nominal dense TF32 1.1 PFLOP/s
    # one CTA alone runs its SM's share of the rate
    ops, ms = fmmbem_peak(FMMBEM_PEAK_TF32, 4000, blocks=1)
    assert ops / (ms * 1e-3) < rate[FMMBEM_PEAK_TF32] / sms * 1.5
