"""CPU checks of the C ABI: the library loads, exports every declared entry point,
and its host-side relaxation rule makes exactly the oracle's decisions."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libfmm():
    from paper_1506_05957_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fmmbem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmmbem_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fmmbem_create", "fmmbem_matvec", "fmmbem_solve", "fmmbem_destroy", "fmmbem_rhs",
                     "fmmbem_n_unknowns", "fmmbem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libfmm):
    missing = [n for n in declared_functions() if not hasattr(libfmm, n)]
    assert not missing, missing


def test_relaxed_p_matches_oracle_bit_for_bit(libfmm):
    from oracle.schedule import relaxed_p
    from paper_1506_05957_gb300 import fmmbem_relaxed_p
    rng = np.random.default_rng(0)
    etas = 10.0 ** rng.uniform(-12, -1, 400)
    rhos = 10.0 ** rng.uniform(-14, 1, 400)
    for eta, rho in zip(etas, rhos):
        for pi, pm in ((16, 1), (12, 3), (10, 5)):
            assert fmmbem_relaxed_p(eta, rho, pi, pm) == relaxed_p(eta, rho, pi, pm)
    # exact powers of two sit on the boundary of the ceiling
    for k in range(1, 40):
        assert fmmbem_relaxed_p(2.0 ** -k, 1.0, 64, 0) == relaxed_p(2.0 ** -k, 1.0, 64, 0) == k


def test_default_opts(libfmm):
    from paper_1506_05957_gb300 import fmmbem_default_opts
    o = fmmbem_default_opts()
    assert (o.p_max, o.restart, o.max_iter, o.near_factor, o.mu) == (16, 50, 100, 2.0, 1.0)


def test_create_rejects_bad_arguments_without_touching_the_gpu(libfmm):
    # argument validation happens before any CUDA call
    from paper_1506_05957_gb300 import binding
    h = ctypes.c_void_p()
    rc = binding.lib().fmmbem_create(None, 0, 4, 150, 0.5, None, ctypes.byref(h))
    assert rc == binding.FMMBEM_EINVAL and not h.value
    v = np.zeros((3, 3))
    t = np.array([[0, 1, 2]], dtype=np.int32)
    mesh = binding.fmmbem_mesh(3, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1,
                               t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    empty = binding.fmmbem_mesh(3, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0,
                                t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    rc = binding.lib().fmmbem_create(ctypes.byref(empty), 0, 4, 150, 0.5, None, ctypes.byref(h))
    assert rc == binding.FMMBEM_EINVAL and not h.value  # an empty mesh is refused
    for kernel, k, ncrit, theta in ((7, 4, 150, 0.5), (0, 4, 150, 1.5), (0, 4, 150, 0.0), (0, 4, 2, 0.5)):
        rc = binding.lib().fmmbem_create(ctypes.byref(mesh), kernel, k, ncrit, theta, None, ctypes.byref(h))
        assert rc == binding.FMMBEM_EINVAL
        assert binding.lib().fmmbem_last_error().decode()


def test_create_rejects_bad_near_rule_and_bodies(libfmm):
    # near_k outside the collapsed products and body indices out of range are refused before any CUDA call
    from paper_1506_05957_gb300 import binding
    from synth import icosphere
    v, t = icosphere(1)
    v = np.ascontiguousarray(v)
    t = np.ascontiguousarray(t, dtype=np.int32)
    mesh = binding.fmmbem_mesh(len(v), v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t),
                               t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    h = ctypes.c_void_p()
    for nk in (7, 20 + 1, 56, -2):
        o = binding.fmmbem_default_opts()
        o.near_k = nk
        rc = binding.lib().fmmbem_create(ctypes.byref(mesh), 0, 4, 150, 0.5, ctypes.byref(o), ctypes.byref(h))
        assert rc == binding.FMMBEM_EINVAL and not h.value
        assert b"near_k" in binding.lib().fmmbem_last_error()
    body = np.zeros(len(t), dtype=np.int32)
    body[3] = 2
    mesh.n_bodies = 2
    mesh.body_of_panel = body.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    rc = binding.lib().fmmbem_create(ctypes.byref(mesh), 0, 4, 150, 0.5, None, ctypes.byref(h))
    assert rc == binding.FMMBEM_EINVAL and b"body_of_panel" in binding.lib().fmmbem_last_error()
    mesh.body_of_panel = None
    rc = binding.lib().fmmbem_create(ctypes.byref(mesh), 0, 4, 150, 0.5, None, ctypes.byref(h))
    assert rc == binding.FMMBEM_EINVAL and not h.value
