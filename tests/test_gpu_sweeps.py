"""The harness of the paper's parameter studies (bench.py --problem sweeps), run on small
meshes (--quick): one JSON line per study, and the relations the paper reports hold in it -
relaxed and non-relaxed solves take the same number of iterations within one (Sec. 3.1),
refined solves meet tolerances below the mixed-precision floor, the Stokes p_min study
converges down to p_min = 3 (Table stokes_min_p), and the Richardson numbers of the cell
drag are those of the oracle's pinned routine applied to the reported drags."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sweep_harness_quick():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import richardson
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--problem", "sweeps", "--quick"],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]
    by = {l["study"]: l for l in lines}
    assert set(by) == {"initial_p", "tolerance", "p_min", "rbc_richardson", "rbc_single_cell"}
    for row in by["initial_p"]["rows"]:
        assert row["iters"] == 10 and row["p_hist"][0] == row["p_initial"]
    tol_rows = by["tolerance"]["rows"]
    assert {r["precision"] for r in tol_rows} == {"mixed", "refined", "fp64"}
    for r in tol_rows:
        assert r["converged"], r
        assert abs(r["iters_relaxed"] - r["iters_fixed"]) <= 1, r
        assert r["true_res"] <= r["tol"] * (1.0 + 1e-6), r
    assert min(r["tol"] for r in tol_rows if r["precision"] == "refined") <= 1e-10
    for r in by["p_min"]["rows"]:
        if r["p_min"] >= 3:
            assert r["converged"] and r["drag_error"] < 5e-2, r
    rr = by["rbc_richardson"]
    f1, f2, f3 = rr["drag"]
    assert f1 < 0 and f2 < 0 and f3 < 0
    assert abs(rr["extrapolated"] - richardson.extrapolate(f1, f2, f3)) <= 1e-12 * abs(rr["extrapolated"])
    assert abs(rr["observed_order"] - richardson.observed_order(f1, f2, f3, 4.0)) <= 1e-12
    for r in by["rbc_single_cell"]["rows"]:
        assert abs(r["iters_relaxed"] - r["iters_fixed"]) <= 2, r
