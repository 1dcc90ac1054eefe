"""ctypes binding of libfmmbem.so, the C ABI declared in include/fmmbem.h.

Argument marshalling only: every step of the mat-vec and the solve runs in the
library's CUDA kernels. Device buffers are passed as torch CUDA tensors (float64,
contiguous); host buffers as numpy arrays. If the library has not been built,
loading raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfmmbem.so")

FMMBEM_OK = 0
FMMBEM_NOT_CONVERGED = 1
FMMBEM_EINVAL = -1
FMMBEM_ENOMEM = -2
FMMBEM_EDEVICE = -3
FMMBEM_ENAN = -4
FMMBEM_ESTATE = -5
FMMBEM_ETIMEOUT = -6
FMMBEM_LAPLACE = 0
FMMBEM_STOKES = 1
FMMBEM_FP64 = 0
FMMBEM_MIXED = 1
FMMBEM_MIXED_REFINED = 2
FMMBEM_P_MAX = 16
FMMBEM_M2L_TABLES = 0
FMMBEM_M2L_GATHER = 1
FMMBEM_M2L_TENSOR = 2
FMMBEM_LAYER_SINGLE = 0
FMMBEM_LAYER_DOUBLE = 1
PASS_NAMES = ["p2m", "m2m", "m2l", "l2l", "l2p", "p2p", "krylov", "matvec"]
FMMBEM_PEAK_FFMA = 0
FMMBEM_PEAK_FFMA2 = 1
FMMBEM_PEAK_RSQRT = 2
FMMBEM_PEAK_DFMA = 3
FMMBEM_PEAK_TF32 = 4


class fmmbem_mesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("vertices", ctypes.POINTER(ctypes.c_double)),
                ("n_panels", ctypes.c_int64), ("triangles", ctypes.POINTER(ctypes.c_int32)),
                ("n_bodies", ctypes.c_int32), ("body_of_panel", ctypes.POINTER(ctypes.c_int32))]


class fmmbem_opts(ctypes.Structure):
    _fields_ = [("p_max", ctypes.c_int), ("near_factor", ctypes.c_double), ("mu", ctypes.c_double),
                ("precision", ctypes.c_int), ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("near_k", ctypes.c_int)]


class fmmbem_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_panels", "n_sources", "n_cells", "n_leaves", "n_levels",
                                               "n_m2l_pairs", "n_m2l_same_level", "n_p2p_pairs",
                                               "n_p2p_interactions", "n_corrections", "n_m2l_tables", "n_m2l_tiles")] + \
               [("setup_seconds", ctypes.c_double), ("n_m2l_tiles_tc", ctypes.c_int64)]


class fmmbem_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8), ("calls", ctypes.c_int64 * 8),
                ("m2l_flops", ctypes.c_double), ("p2p_interactions", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("tc_ms", ctypes.c_double), ("tc_flops", ctypes.c_double)]


class fmmbem_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("true_res", ctypes.c_double), ("queue_s", ctypes.c_double), ("setup_s", ctypes.c_double),
                ("solve_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("handle_reused", ctypes.c_int32)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def lib():
    """The loaded library; raises if it was not built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfmmbem.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.fmmbem_default_opts.argtypes = [ctypes.POINTER(fmmbem_opts)]
        L.fmmbem_create.argtypes = [ctypes.POINTER(fmmbem_mesh), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.POINTER(fmmbem_opts), ctypes.POINTER(_vp)]
        L.fmmbem_destroy.argtypes = [_vp]
        L.fmmbem_destroy.restype = None
        L.fmmbem_n_unknowns.argtypes = [_vp]
        L.fmmbem_n_unknowns.restype = ctypes.c_int64
        L.fmmbem_set_precision.argtypes = [_vp, ctypes.c_int]
        L.fmmbem_matvec.argtypes = [_vp, ctypes.c_int, _vp, _vp]
        L.fmmbem_set_m2l_mode.argtypes = [_vp, ctypes.c_int]
        L.fmmbem_set_p2p_variant.argtypes = [_vp, ctypes.c_int]
        L.fmmbem_set_device_loop.argtypes = [_vp, ctypes.c_int]
        L.fmmbem_set_layer.argtypes = [_vp, ctypes.c_int]
        L.fmmbem_solve_batch.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                         _vp, _vp, _vp]
        L.fmmbem_set_tc_thresholds.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
        L.fmmbem_autotune.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp]
        L.fmmbem_estimate_bytes.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(fmmbem_opts)]
        L.fmmbem_estimate_bytes.restype = ctypes.c_int64
        L.fmmbem_server_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(_vp)]
        L.fmmbem_server_submit.argtypes = [_vp, ctypes.POINTER(fmmbem_mesh), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.POINTER(fmmbem_opts), _dp, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                           ctypes.POINTER(ctypes.c_int64)]
        L.fmmbem_server_wait.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(fmmbem_result)]
        L.fmmbem_server_destroy.argtypes = [_vp]
        L.fmmbem_server_set_cache.argtypes = [_vp, ctypes.c_int]
        L.fmmbem_server_cache_hits.argtypes = [_vp]
        L.fmmbem_server_cache_hits.restype = ctypes.c_int64
        L.fmmbem_matvec_direct.argtypes = [_vp, _vp, _vp]
        L.fmmbem_rhs.argtypes = [_vp, _vp, _vp]
        L.fmmbem_stokes_dl_apply.argtypes = [_vp, _vp, _vp]
        L.fmmbem_relaxed_p.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.fmmbem_solve.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                   ctypes.POINTER(ctypes.c_int), _vp, _vp, _dp]
        L.fmmbem_solve_host.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                        ctypes.POINTER(ctypes.c_int), _vp, _vp, _dp]
        L.fmmbem_expansion_eval.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int, _vp,
                                            ctypes.c_int, _vp, _vp, _vp]
        L.fmmbem_expansion_eval_static.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int,
                                                   _vp, ctypes.c_int, _vp, _vp, _vp]
        L.fmmbem_get_stats.argtypes = [_vp, ctypes.POINTER(fmmbem_stats)]
        L.fmmbem_profile_enable.argtypes = [_vp, ctypes.c_int]
        L.fmmbem_profile_get.argtypes = [_vp, ctypes.POINTER(fmmbem_profile)]
        L.fmmbem_last_error.restype = ctypes.c_char_p
        L.fmmbem_create_tuned.argtypes = [ctypes.POINTER(fmmbem_mesh), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.POINTER(fmmbem_opts),
                                          ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int),
                                          _dp]
        L.fmmbem_body_integrals.argtypes = [_vp, _vp, _vp]
        L.fmmbem_n_bodies.argtypes = [_vp]
        L.fmmbem_check_waits.argtypes = [_vp]
        L.fmmbem_set_wait_limit.argtypes = [_vp, ctypes.c_uint]
        L.fmmbem_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _vp]
        L.fmmbem_sort_pairs_u64.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, _vp]
        L.fmmbem_scan_i32.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int, _vp]
        _lib = L
    return _lib


class FmmBemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fmmbem error %d: %s" % (code, msg))
        self.code = code


def _check(rc):
    if rc < 0:
        raise FmmBemError(rc, lib().fmmbem_last_error().decode())
    return rc


def _dev(t, n=None):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, t.numel()))
    return _vp(t.data_ptr())


def _host(a, n):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == n):
        raise TypeError("expected a contiguous float64 numpy array of %d elements" % n)
    return _vp(a.ctypes.data)


def fmmbem_default_opts():
    o = fmmbem_opts()
    _check(lib().fmmbem_default_opts(ctypes.byref(o)))
    return o


def fmmbem_relaxed_p(eta, rho_prev, p_initial, p_min):
    return int(lib().fmmbem_relaxed_p(float(eta), float(rho_prev), int(p_initial), int(p_min)))


def fmmbem_expansion_eval(kind, p, center, scale, src, tgt, out, stream=None):
    """src: [n,4] (x,y,z,q) CUDA float64; tgt: [m,3]; out: [m]."""
    c = (ctypes.c_double * 3)(*[float(v) for v in center])
    _check(lib().fmmbem_expansion_eval(int(kind), int(p), c, float(scale), int(src.shape[0]), _dev(src),
                                       int(tgt.shape[0]), _dev(tgt), _dev(out), _vp(stream)))


def fmmbem_expansion_eval_static(kind, p, center, scale, src, tgt, out, stream=None):
    """Allocation-free fmmbem_expansion_eval (fixed module-global scratch; asynchronous)."""
    c = (ctypes.c_double * 3)(*[float(v) for v in center])
    _check(lib().fmmbem_expansion_eval_static(int(kind), int(p), c, float(scale), int(src.shape[0]), _dev(src),
                                              int(tgt.shape[0]), _dev(tgt), _dev(out), _vp(stream)))


def fmmbem_peak(kind, iters, blocks=0, stream=None):
    """fmmbem_peak: (operations, milliseconds) of one peak-rate launch (synchronizes the stream)."""
    ops, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().fmmbem_peak(int(kind), int(blocks), int(iters), ctypes.byref(ops), ctypes.byref(ms), _vp(stream)))
    return ops.value, ms.value


def _dev_typed(t, dtype, what):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("expected a contiguous %s CUDA tensor for %s" % (dtype, what))
    return _vp(t.data_ptr())


def sort_pairs_u64(keys, values=None, end_bit=0, stream=None):
    """fmmbem_sort_pairs_u64: (sorted keys, their values) of int64 CUDA tensors whose bits are the
    unsigned 64-bit keys; values (int32, optional) follow their keys, equal keys keep their order."""
    import torch
    n = int(keys.numel())
    kout = torch.empty_like(keys)
    kp = _dev_typed(keys, torch.int64, "keys") if n else None
    vout = torch.empty_like(values) if values is not None else None
    vp = _dev_typed(values, torch.int32, "values") if (values is not None and n) else None
    if values is not None and values.numel() != n:
        raise ValueError("one value per key")
    _check(lib().fmmbem_sort_pairs_u64(kp, _vp(kout.data_ptr()) if n else None, vp,
                                       _vp(vout.data_ptr()) if (vp is not None) else None, n, int(end_bit), _vp(stream)))
    return kout, vout


def scan_i32(x, inclusive=False, out=None, stream=None):
    """fmmbem_scan_i32: exclusive (or inclusive) prefix sum of an int32 CUDA tensor."""
    import torch
    n = int(x.numel())
    out = torch.empty_like(x) if out is None else out
    ip = _dev_typed(x, torch.int32, "input") if n else None
    op = _dev_typed(out, torch.int32, "output") if n else None
    _check(lib().fmmbem_scan_i32(ip, op, n, 1 if inclusive else 0, _vp(stream)))
    return out


class FmmBem:
    """One resident BEM problem: fmmbem_create ... fmmbem_destroy."""

    def __init__(self, vertices, triangles, kernel=FMMBEM_LAPLACE, gauss_k=4, ncrit=150, theta=0.5, p_max=16,
                 near_factor=2.0, mu=1.0, precision=FMMBEM_MIXED, restart=50, max_iter=100, stream=None, nrhs=1,
                 near_k=20, body_of_panel=None, _tune=None):
        """_tune = (ncrit candidates, p_lo, p_hi): create through fmmbem_create_tuned (see FmmBem.tuned)."""
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        t = np.ascontiguousarray(triangles, dtype=np.int32)
        mesh = fmmbem_mesh(len(v), v.ctypes.data_as(_dp), len(t), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if body_of_panel is not None:
            bop = np.ascontiguousarray(body_of_panel, dtype=np.int32)
            if bop.shape != (len(t),):
                raise ValueError("body_of_panel needs one entry per panel")
            mesh.n_bodies = int(bop.max()) + 1 if len(bop) else 0
            mesh.body_of_panel = bop.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        o = fmmbem_default_opts()
        o.p_max, o.near_factor, o.mu, o.precision = p_max, near_factor, mu, precision
        o.restart, o.max_iter = restart, max_iter
        o.nrhs = nrhs
        o.near_k = near_k
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        o.stream = stream
        h = _vp()
        self.tuned_ncrit, self.tuned_ms = None, None
        if _tune is None:
            _check(lib().fmmbem_create(ctypes.byref(mesh), int(kernel), int(gauss_k), int(ncrit), float(theta),
                                       ctypes.byref(o), ctypes.byref(h)))
        else:
            cand, p_lo, p_hi = _tune
            arr = (ctypes.c_int * len(cand))(*[int(c) for c in cand])
            nc, ms = ctypes.c_int(0), ctypes.c_double(0.0)
            _check(lib().fmmbem_create_tuned(ctypes.byref(mesh), int(kernel), int(gauss_k), len(cand), arr,
                                             float(theta), ctypes.byref(o), int(p_lo), int(p_hi), ctypes.byref(h),
                                             ctypes.byref(nc), ctypes.byref(ms)))
            self.tuned_ncrit, self.tuned_ms = nc.value, ms.value
        self.h = h
        self.kernel = kernel
        self.max_iter = max_iter
        self.nrhs = int(nrhs)
        self.p_max = int(p_max)
        self.n = int(lib().fmmbem_n_unknowns(h)) * self.nrhs  # doubles per mat-vec vector (all of a batch)
        self.n_panels = len(t)
        self.n_bodies = int(lib().fmmbem_n_bodies(h))

    @classmethod
    def tuned(cls, vertices, triangles, ncrit_candidates=(100, 125, 150, 175, 200), p_lo=3, p_hi=12, **kw):
        """fmmbem_create_tuned: the leaf capacity (and per-order kernel choices) picked by timing mat-vecs
        over [p_lo, p_hi]; .tuned_ncrit holds the choice."""
        return cls(vertices, triangles, _tune=(tuple(ncrit_candidates), p_lo, p_hi), **kw)

    def close(self):
        if getattr(self, "h", None):
            lib().fmmbem_destroy(self.h)
            self.h = None

    __del__ = close

    def set_precision(self, precision):
        _check(lib().fmmbem_set_precision(self.h, int(precision)))

    def set_layer(self, layer):
        """FMMBEM_LAYER_SINGLE (A = V) or FMMBEM_LAYER_DOUBLE (A = 1/2 I + K) for later mat-vecs and solves."""
        _check(lib().fmmbem_set_layer(self.h, int(layer)))

    def set_tc_thresholds(self, m2l_min_p, tree_min_p):
        """Lowest p at which M2L and M2M/L2L run on the tensor cores (mixed precision)."""
        _check(lib().fmmbem_set_tc_thresholds(self.h, int(m2l_min_p), int(tree_min_p)))

    def autotune(self, p_lo=1, p_hi=None):
        """fmmbem_autotune: near-field schedule (key 0) and per-order choice of tensor-core or SIMT M2L and
        M2M/L2L; returns {0: p2p variant, p: choice}."""
        p_hi = self.p_max if p_hi is None else p_hi
        ch = np.full(FMMBEM_P_MAX + 1, -1, dtype=np.int32)
        _check(lib().fmmbem_autotune(self.h, int(p_lo), int(p_hi), _vp(ch.ctypes.data)))
        out = {0: int(ch[0])}
        out.update({p: int(ch[p]) for p in range(p_lo, p_hi + 1)})
        return out

    def body_integrals(self, x):
        """fmmbem_body_integrals: [n_bodies, dof] sums of S_j x_j over each body's panels (Stokes traction
        -> force on each body)."""
        dof = 3 if self.kernel == FMMBEM_STOKES else 1
        out = np.zeros((self.n_bodies, dof), dtype=np.float64)
        _check(lib().fmmbem_body_integrals(self.h, _dev(x, self.n // self.nrhs), _vp(out.ctypes.data)))
        return out

    def check_waits(self):
        """fmmbem_check_waits: raises FmmBemError(FMMBEM_ETIMEOUT) if a bounded device wait of the work
        queued since the last check gave up (mat-vecs do not report it themselves)."""
        _check(lib().fmmbem_check_waits(self.h))

    def set_wait_limit(self, limit):
        """Test hook: polls before a grid-barrier wait of the Arnoldi step gives up (0 = default)."""
        _check(lib().fmmbem_set_wait_limit(self.h, int(limit)))

    def set_p2p_variant(self, variant):
        _check(lib().fmmbem_set_p2p_variant(self.h, int(variant)))

    def set_device_loop(self, on=True):
        """Run each GMRES restart cycle as one device-resident graph (fmmbem_set_device_loop)."""
        _check(lib().fmmbem_set_device_loop(self.h, 1 if on else 0))

    def set_m2l_mode(self, mode):
        _check(lib().fmmbem_set_m2l_mode(self.h, int(mode)))

    def matvec(self, p, x, y):
        _check(lib().fmmbem_matvec(self.h, int(p), _dev(x, self.n), _dev(y, self.n)))

    def matvec_direct(self, x, y):
        _check(lib().fmmbem_matvec_direct(self.h, _dev(x, self.n), _dev(y, self.n)))

    def rhs(self, known, b):
        m = self.n_panels * self.nrhs
        _check(lib().fmmbem_rhs(self.h, _dev(known, m), _dev(b, m)))

    def stokes_dl_apply(self, u, y):
        _check(lib().fmmbem_stokes_dl_apply(self.h, _dev(u, self.n), _dev(y, self.n)))

    def _solve(self, fn, b, x, tol, relax, p_initial, p_min):
        it = ctypes.c_int(0)
        ph = np.zeros(self.max_iter + 1, dtype=np.int32)
        rh = np.zeros(self.max_iter + 2, dtype=np.float64)
        tr = ctypes.c_double(0.0)
        rc = _check(fn(self.h, b, float(tol), int(bool(relax)), int(p_initial), int(p_min), x, ctypes.byref(it),
                       _vp(ph.ctypes.data), _vp(rh.ctypes.data), ctypes.byref(tr)))
        k = it.value
        return dict(converged=(rc == 0), iters=k, p_hist=ph[:k].tolist(), res_hist=rh[:k + 1].tolist(),
                    true_res=tr.value)

    def solve_batch(self, b, x, tol=1e-6, relax=True, p_initial=10, p_min=3):
        """fmmbem_solve_batch: b, x are [nrhs * n_panels] device tensors (vector q at q * n_panels)."""
        nb = self.nrhs
        it = np.zeros(nb, dtype=np.int32)
        ph = np.zeros(self.max_iter + 1, dtype=np.int32)
        rh = np.zeros(nb * (self.max_iter + 1), dtype=np.float64)
        tr = np.zeros(nb, dtype=np.float64)
        rc = _check(lib().fmmbem_solve_batch(self.h, _dev(b, self.n), float(tol), int(bool(relax)), int(p_initial),
                                             int(p_min), _dev(x, self.n), _vp(it.ctypes.data), _vp(ph.ctypes.data),
                                             _vp(rh.ctypes.data), _vp(tr.ctypes.data)))
        return dict(converged=(rc == 0), iters=it.tolist(), p_hist=ph[:int(it.max())].tolist(),
                    res_hist=[rh[q * (self.max_iter + 1):q * (self.max_iter + 1) + it[q] + 1].tolist()
                              for q in range(nb)], true_res=tr.tolist())

    def solve(self, b, x, tol=1e-6, relax=True, p_initial=10, p_min=3):
        return self._solve(lib().fmmbem_solve, _dev(b, self.n), _dev(x, self.n), tol, relax, p_initial, p_min)

    def solve_host(self, b, x, tol=1e-6, relax=True, p_initial=10, p_min=3):
        return self._solve(lib().fmmbem_solve_host, _host(b, self.n), _host(x, self.n), tol, relax, p_initial, p_min)

    def stats(self):
        s = fmmbem_stats()
        _check(lib().fmmbem_get_stats(self.h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in fmmbem_stats._fields_}

    def profile_enable(self, on=True):
        """fmmbem_profile_enable: 0 off, 1 (True) the solve's own schedule, 2 passes serialized."""
        _check(lib().fmmbem_profile_enable(self.h, int(on)))

    def profile(self):
        pr = fmmbem_profile()
        _check(lib().fmmbem_profile_get(self.h, ctypes.byref(pr)))
        return dict(ms={PASS_NAMES[i]: pr.ms[i] for i in range(8)},
                    launches={PASS_NAMES[i]: pr.launches[i] for i in range(8)},
                    calls={PASS_NAMES[i]: pr.calls[i] for i in range(8)},
                    m2l_flops=pr.m2l_flops, p2p_interactions=pr.p2p_interactions,
                    kernel_launches=pr.kernel_launches, tc_ms=pr.tc_ms, tc_flops=pr.tc_flops)


class FmmBemServer:
    """Serving runtime (fmmbem_server_*): solves of different meshes, operators and tolerances
    admitted by an HBM budget and run concurrently by `max_active` worker threads of the library."""

    def __init__(self, max_active=4, hbm_budget=None):
        if hbm_budget is None:
            import torch
            hbm_budget = int(0.8 * torch.cuda.mem_get_info()[0])
        s = _vp()
        _check(lib().fmmbem_server_create(int(max_active), int(hbm_budget), ctypes.byref(s)))
        self.s = s
        self._pending = {}

    def submit(self, vertices, triangles, rhs, kernel=FMMBEM_LAPLACE, gauss_k=4, ncrit=150, theta=0.5, p_max=16,
               mu=1.0, precision=FMMBEM_MIXED, tol=1e-6, relax=True, p_initial=10, p_min=3):
        v = np.ascontiguousarray(vertices, dtype=np.float64)
        t = np.ascontiguousarray(triangles, dtype=np.int32)
        b = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.zeros_like(b)
        mesh = fmmbem_mesh(len(v), v.ctypes.data_as(_dp), len(t), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        o = fmmbem_default_opts()
        o.p_max, o.mu, o.precision = p_max, mu, precision
        tk = ctypes.c_int64()
        _check(lib().fmmbem_server_submit(self.s, ctypes.byref(mesh), int(kernel), int(gauss_k), int(ncrit),
                                          float(theta), ctypes.byref(o), b.ctypes.data_as(_dp), float(tol),
                                          int(bool(relax)), int(p_initial), int(p_min), x.ctypes.data_as(_dp),
                                          ctypes.byref(tk)))
        self._pending[tk.value] = x  # the library writes the solution here
        return tk.value

    def wait(self, ticket):
        r = fmmbem_result()
        _check(lib().fmmbem_server_wait(self.s, int(ticket), ctypes.byref(r)))
        x = self._pending.pop(ticket)
        return x, {n: getattr(r, n) for n, _ in fmmbem_result._fields_}

    def set_cache(self, max_handles):
        """fmmbem_server_set_cache: keep at most max_handles idle handles (0: no cache)."""
        _check(lib().fmmbem_server_set_cache(self.s, int(max_handles)))

    def cache_hits(self):
        return int(lib().fmmbem_server_cache_hits(self.s))

    def close(self):
        if getattr(self, "s", None):
            lib().fmmbem_server_destroy(self.s)
            self.s = None

    __del__ = close


def fmmbem_estimate_bytes(n_panels, kernel=FMMBEM_LAPLACE, gauss_k=4, ncrit=150, p_max=16):
    o = fmmbem_default_opts()
    o.p_max = p_max
    return lib().fmmbem_estimate_bytes(int(n_panels), int(kernel), int(gauss_k), int(ncrit), ctypes.byref(o))
