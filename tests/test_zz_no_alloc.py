"""Allocation-free expansion evaluation (fmmbem_expansion_eval_static).

Callers that cannot allocate device memory (graph capture, arenas, real-time loops)
use this entry point; it must give the same numbers as fmmbem_expansion_eval, call
after call, although every call reuses the same fixed scratch array. Collected last
so a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_scratch_matches_allocating_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_05957_gb300 import build
    build.build()
    from paper_1506_05957_gb300.binding import lib

    L = lib()
    rng = np.random.default_rng(11)

    def case(kind, p, n_src, n_tgt, center, scale):
        if kind == 0:  # sources near the centre, targets far away
            src = center + 0.3 * (rng.random((n_src, 3)) - 0.5)
            d = rng.standard_normal((n_tgt, 3))
            tgt = center + 1.5 * d / np.linalg.norm(d, axis=1)[:, None]
        else:  # sources far away, targets near the centre
            d = rng.standard_normal((n_src, 3))
            src = center + 2.0 * d / np.linalg.norm(d, axis=1)[:, None]
            tgt = center + 0.3 * (rng.random((n_tgt, 3)) - 0.5)
        s = torch.tensor(np.column_stack([src, rng.standard_normal(n_src)]), dtype=torch.float64, device="cuda")
        t = torch.tensor(tgt, dtype=torch.float64, device="cuda")
        return s, t

    c = (ctypes.c_double * 3)
    calls = [(0, 12, 300, 257, np.array([0.1, -0.2, 0.3]), 0.5),
             (1, 16, 200, 130, np.array([-1.0, 0.5, 0.0]), 1.7)]
    for kind, p, ns, nt, center, scale in calls:  # two calls in a row, different sizes and orders
        src, tgt = case(kind, p, ns, nt, center, scale)
        ref = torch.zeros(nt, dtype=torch.float64, device="cuda")
        out = torch.full((nt,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.fmmbem_expansion_eval(kind, p, c(*center), scale, ns, ctypes.c_void_p(src.data_ptr()), nt,
                                     ctypes.c_void_p(tgt.data_ptr()), ctypes.c_void_p(ref.data_ptr()), None)
        assert rc == 0, L.fmmbem_last_error()
        rc = L.fmmbem_expansion_eval_static(kind, p, c(*center), scale, ns, ctypes.c_void_p(src.data_ptr()), nt,
                                            ctypes.c_void_p(tgt.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, L.fmmbem_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - r)) <= 1e-12 * np.max(np.abs(r))

    # sizes beyond the scratch are refused with a message, before any GPU work
    src, tgt = case(0, 4, 8, 8, np.zeros(3), 1.0)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.fmmbem_expansion_eval_static(0, 17, c(0, 0, 0), 1.0, 8, ctypes.c_void_p(src.data_ptr()), 8,
                                        ctypes.c_void_p(tgt.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1 and b"static scratch" in L.fmmbem_last_error()
