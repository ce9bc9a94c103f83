"""Python binding of the GB300 IIM Poisson solver library (``_lib/libiim.so``).

Argument marshalling only: every computation runs in the CUDA kernels behind
the C ABI declared in ``include/iim.h``.  PyTorch provides device memory and
streams.  Importing this module does not need a GPU; creating a problem does,
and fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libiim.so")

IIM_OK = 0
IIM_ERR_INVALID_ARG, IIM_ERR_CURVATURE, IIM_ERR_RANK, IIM_ERR_SINGULAR = 1, 2, 3, 4
IIM_ERR_NOT_CONVERGED, IIM_ERR_BREAKDOWN, IIM_ERR_BUDGET, IIM_ERR_TIMEOUT = 5, 6, 7, 8
IIM_ERR_CUDA, IIM_ERR_GEOMETRY, IIM_ERR_CAPACITY = 9, 10, 11
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "curvature", 3: "rank", 4: "singular", 5: "not converged",
                6: "breakdown", 7: "budget", 8: "timeout", 9: "cuda", 10: "geometry", 11: "capacity"}
GEOM = {"circle": 0, "ellipse": 1, "star": 2, "sphere": 3, "ellipsoid": 4, "perturbed_sphere": 5, "fourier": 6,
        "levelset_grid": 7}
MAX_FOURIER_MODES = 16
BC = {"dirichlet": 0, "neumann": 1, "interface": 2}
MG_FP32, MG_FP64, MG_FP32_BF16R = 0, 1, 2
CYCLE_V, CYCLE_W = 1, 2
KRYLOV_FGMRES, KRYLOV_GMRES_LEFT = 0, 1


class IIMError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"iim status {status} ({STATUS_NAMES.get(status, '?')}): {msg}")


class Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("geom_kind", ctypes.c_int),
                ("plus_inside", ctypes.c_int), ("geom_params", ctypes.c_double * 8), ("bc", ctypes.c_int),
                ("box_bc", ctypes.c_int), ("beta_plus", ctypes.c_double), ("beta_minus", ctypes.c_double),
                ("order", ctypes.c_int), ("geom_coef", ctypes.c_void_p), ("n_geom_coef", ctypes.c_int),
                ("phi_dev", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("mg_precision", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("reorth", ctypes.c_int), ("cycle", ctypes.c_int),
                ("krylov", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("relres", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("kernels", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

SIGNATURES = {
    "iim_default_options": (None, [ctypes.POINTER(Options)]),
    "iim_problem_create": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.POINTER(Options), ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "iim_problem_setup": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iim_status_get": (ctypes.c_int, [ctypes.c_void_p]),
    "iim_problem_destroy": (None, [ctypes.c_void_p]),
    "iim_problem_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "iim_control_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iim_problem_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "iim_problem_fit_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]),
    "iim_phase": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iim_control_point_edges": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iim_box_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iim_problem_set_phi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iim_set_data": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5),
    "iim_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "iim_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iim_boundary_values": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iim_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iim_apply_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "iim_precondition": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "iim_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(SolveInfo)]),
    "iim_solve_host": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.POINTER(SolveInfo)]),
    "iim_batch_solve": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.POINTER(SolveInfo)]),
    "iim_kernel_time": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "iim_kernel_time_flushed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)]),
    "iim_launch_count": (ctypes.c_int64, []),
    "iim_engine_create": (ctypes.c_int, [ctypes.POINTER(Options), ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "iim_engine_destroy": (None, [ctypes.c_void_p]),
    "iim_engine_admit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "iim_engine_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "iim_engine_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "iim_engine_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(SolveInfo)]),
    "iim_engine_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "iim_engine_set_shapes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "iim_engine_get_shapes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "iim_engine_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "iim_server_create": (ctypes.c_int, [ctypes.POINTER(Options), ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "iim_server_destroy": (None, [ctypes.c_void_p]),
    "iim_server_set_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "iim_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_int64)]),
    "iim_server_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "iim_server_problem": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int64]),
    "iim_server_data_ready": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "iim_server_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "iim_server_take": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(SolveInfo),
                                       ctypes.POINTER(ctypes.c_double)]),
    "iim_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                        ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "iim_server_set_pooling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "iim_server_pool_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int)]),
    "iim_last_error": (ctypes.c_char_p, []),
    "iim_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path: str = LIB_PATH):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"IIM CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, what=""):
    if status != IIM_OK:
        msg = load().iim_last_error().decode(errors="replace")
        raise IIMError(status, f"{what}: {msg}")


def default_options(**kw) -> Options:
    o = Options()
    load().iim_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_desc(dim, n, geom_kind, geom_params, plus_inside, bc, box_bc, beta_plus=1.0, beta_minus=1.0, order=4,
              coef=None, phi=None):
    """``coef``: the Fourier curve's a0, a1, b1, ... (host); ``phi``: a contiguous float64 CUDA
    tensor of the level set at the grid's nodes (x0 fastest).  The descriptor keeps both
    alive (they are read when the problem is created)."""
    d = Desc()
    d.dim, d.n, d.geom_kind, d.plus_inside = int(dim), int(n), int(geom_kind), int(bool(plus_inside))
    p = list(geom_params) + [0.0] * (8 - len(geom_params))
    for k in range(8):
        d.geom_params[k] = float(p[k])
    d.bc, d.box_bc = int(bc), int(box_bc)
    d.beta_plus, d.beta_minus = float(beta_plus), float(beta_minus)
    d.order = int(order)
    d._keep = []
    if coef is not None and len(coef):
        arr = (ctypes.c_double * len(coef))(*[float(v) for v in coef])
        d._keep.append(arr)
        d.geom_coef = ctypes.cast(arr, ctypes.c_void_p)
        d.n_geom_coef = len(coef)
    if phi is not None:
        d._keep.append(phi)
        d.phi_dev = _ptr(phi)
    return d


def desc_from_spec(spec) -> Desc:
    """Descriptor from any object with the fields of a problem statement (n, geometry, bc, ...)."""
    g = spec.geometry
    phi = None
    if g.kind == GEOM["levelset_grid"]:
        import numpy as np
        import torch
        phi = torch.as_tensor(np.ascontiguousarray(np.asarray(g.values).ravel(order="F")), dtype=torch.float64,
                              device="cuda")
    return make_desc(g.dim, spec.n, g.kind, g.params, g.plus_inside, spec.bc, spec.box_bc,
                     spec.beta_plus, spec.beta_minus, spec.order, coef=getattr(g, "coef", None), phi=phi)


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    """Host buffer pointer (numpy array or pinned/pageable CPU tensor of float64)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    import numpy as np
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


class Problem:
    """One immersed-interface Poisson problem resident on the device."""

    def __init__(self, desc: Desc, options: Options | None = None, stream=None):
        import torch
        lib = load()
        self.desc = desc
        self.options = options or default_options()
        self.stream = stream or torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = lib.iim_problem_create(ctypes.byref(desc), ctypes.byref(self.options),
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(st, "iim_problem_create")
        self.h = h
        K, B = ctypes.c_int(), ctypes.c_int()
        N, U = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.iim_problem_sizes(self.h, ctypes.byref(K), ctypes.byref(B), ctypes.byref(N), ctypes.byref(U)))
        self.K, self.B, self.N, self.n_unknowns = K.value, B.value, N.value, U.value
        self.dim, self.n = desc.dim, desc.n

    @classmethod
    def view(cls, handle, desc: Desc):
        """A non-owning view of a problem the library holds (e.g. a server request)."""
        self = cls.__new__(cls)
        lib = load()
        self.desc, self.options, self.stream, self._owned = desc, None, None, False
        self.h = ctypes.c_void_p(handle)
        K, B = ctypes.c_int(), ctypes.c_int()
        N, U = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.iim_problem_sizes(self.h, ctypes.byref(K), ctypes.byref(B), ctypes.byref(N), ctypes.byref(U)))
        self.K, self.B, self.N, self.n_unknowns = K.value, B.value, N.value, U.value
        self.dim, self.n = desc.dim, desc.n
        return self

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            load().iim_problem_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *shape, dtype=None):
        import torch
        return torch.empty(*shape, dtype=dtype or torch.float64, device="cuda")

    def setup(self, geom_params=None):
        arr = None
        if geom_params is not None:
            arr = (ctypes.c_double * 8)(*(list(geom_params) + [0.0] * (8 - len(geom_params))))
        _check(load().iim_problem_setup(self.h, arr), "iim_problem_setup")

    def refresh_sizes(self):
        K = ctypes.c_int()
        _check(load().iim_problem_sizes(self.h, ctypes.byref(K), None, None, None))
        self.K = K.value
        return self.K

    def status(self):
        return load().iim_status_get(self.h)

    def device_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(load().iim_problem_bytes(self.h, ctypes.byref(b)))
        return b.value

    def _foreign_stream_sync(self, before):
        """A view's problem runs on a library stream that torch's stream does not order:
        wait for torch's work before the library reads our tensors, and for the
        library's copies before torch reads them."""
        if getattr(self, "_owned", True):
            return
        import torch
        if before:
            torch.cuda.current_stream().synchronize()
        else:
            _check(self.status(), "problem status")

    def control_points(self):
        xc = self._empty(max(self.K, 1), self.dim)
        nc = self._empty(max(self.K, 1), self.dim)
        self._foreign_stream_sync(True)
        _check(load().iim_control_points(self.h, _ptr(xc), _ptr(nc)))
        self._foreign_stream_sync(False)
        return xc[:self.K], nc[:self.K]

    def control_point_edges(self):
        """(axis, lower node, side) of every control point's grid edge (see iim_control_point_edges)."""
        import torch
        ax = torch.empty(max(self.K, 1), dtype=torch.int32, device="cuda")
        lo = torch.empty(max(self.K, 1), dtype=torch.int32, device="cuda")
        sd = torch.empty(max(self.K, 1), dtype=torch.uint8, device="cuda")
        self._foreign_stream_sync(True)
        _check(load().iim_control_point_edges(self.h, ctypes.c_void_p(ax.data_ptr()), ctypes.c_void_p(lo.data_ptr()),
                                              ctypes.c_void_p(sd.data_ptr())), "iim_control_point_edges")
        self._foreign_stream_sync(False)
        return ax[:self.K], lo[:self.K], sd[:self.K]

    def box_points(self):
        """Outer-box Dirichlet sample points, shape (B, dim) (see iim_box_points)."""
        xb = self._empty(max(self.B, 1), self.dim)
        self._foreign_stream_sync(True)
        _check(load().iim_box_points(self.h, _ptr(xb)), "iim_box_points")
        self._foreign_stream_sync(False)
        return xb[:self.B]

    def set_phi(self, phi):
        """Replace a grid level set's node values (then call setup())."""
        self._foreign_stream_sync(True)
        _check(load().iim_problem_set_phi(self.h, _ptr(phi)), "iim_problem_set_phi")

    def phase(self):
        import torch
        ph = torch.empty(self.N, dtype=torch.uint8, device="cuda")
        self._foreign_stream_sync(True)
        _check(load().iim_phase(self.h, ctypes.c_void_p(ph.data_ptr())))
        self._foreign_stream_sync(False)
        return ph

    def set_data(self, f, g=None, j0=None, j1=None, box=None):
        self._foreign_stream_sync(True)
        _check(load().iim_set_data(self.h, _ptr(f), _ptr(g), _ptr(j0), _ptr(j1), _ptr(box)), "iim_set_data")
        # a view's problem reads the tensors on a stream torch does not order: wait for the
        # reads, so that the caller may free or reuse them (from any thread) on return
        self._foreign_stream_sync(False)

    def apply(self, u, include_data=False, out=None):
        w = out if out is not None else self._empty(self.N)
        _check(load().iim_apply(self.h, _ptr(u), _ptr(w), int(include_data)), "iim_apply")
        return w

    def apply_noalloc(self, u, include_data=False, out=None):
        """iim_apply with the ghost values in the library's fixed device area (see iim.h)."""
        w = out if out is not None else self._empty(self.N)
        _check(load().iim_apply_noalloc(self.h, _ptr(u), _ptr(w), int(include_data)), "iim_apply_noalloc")
        return w

    def boundary_values(self, u):
        """Unprescribed boundary quantity at the control points (see iim_boundary_values)."""
        out = self._empty(max(self.K, 1))
        _check(load().iim_boundary_values(self.h, _ptr(u), _ptr(out)), "iim_boundary_values")
        return out[:self.K]

    def gradient(self, u):
        """grad u, shape (dim, N) (see iim_gradient)."""
        g = self._empty(self.dim, self.N)
        _check(load().iim_gradient(self.h, _ptr(u), _ptr(g)), "iim_gradient")
        return g

    def rhs(self):
        b = self._empty(self.N)
        _check(load().iim_rhs(self.h, _ptr(b)))
        return b

    def precondition(self, v, out=None):
        z = out if out is not None else self._empty(self.N)
        _check(load().iim_precondition(self.h, _ptr(v), _ptr(z)), "iim_precondition")
        return z

    def solve(self, x=None, check=True):
        import torch
        if x is None:
            x = torch.zeros(self.N, dtype=torch.float64, device="cuda")
        info = SolveInfo()
        st = load().iim_solve(self.h, _ptr(x), ctypes.byref(info))
        if check:
            _check(st, "iim_solve")
        return x, info

    def solve_host(self, f, g=None, j0=None, j1=None, box=None, x=None, check=True):
        import numpy as np
        if x is None:
            x = np.zeros(self.N)
        info = SolveInfo()
        st = load().iim_solve_host(self.h, _hptr(f), _hptr(g), _hptr(j0), _hptr(j1), _hptr(box), _hptr(x),
                                   ctypes.byref(info))
        if check:
            _check(st, "iim_solve_host")
        return x, info


def batch_solve(problems, xs, check=True):
    lib = load()
    n = len(problems)
    hs = (ctypes.c_void_p * n)(*[p.h.value for p in problems])
    ps = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (SolveInfo * n)()
    st = lib.iim_batch_solve(hs, ps, n, infos)
    if check:
        _check(st, "iim_batch_solve")
    return [infos[i] for i in range(n)], st


KERNELS = {"stencil": 0, "ghost": 1, "correct": 2, "smooth_fine": 3, "multidot": 4, "update": 5, "vcycle": 6,
           "operator": 7, "fits": 8, "mg_down0": 9, "mg_up0": 10, "mg_tail": 11}


def fit_stats(problem):
    """(number of fits, sum of their rows, monomials M) of the problem's current set-up."""
    nf, rs, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(load().iim_problem_fit_stats(problem.h, ctypes.byref(nf), ctypes.byref(rs), ctypes.byref(m)))
    return nf.value, rs.value, m.value


def kernel_time(problem, which, reps=50, flush=None) -> float:
    """Average device microseconds per launch of one internal kernel (see iim_kernel_time);
    with ``flush`` (a device tensor larger than L2) each launch follows an overwrite of it."""
    us = ctypes.c_double()
    if flush is None:
        _check(load().iim_kernel_time(problem.h, KERNELS.get(which, which), int(reps), ctypes.byref(us)),
               "kernel_time")
    else:
        _check(load().iim_kernel_time_flushed(problem.h, KERNELS.get(which, which), int(reps),
                                              ctypes.c_void_p(flush.data_ptr()),
                                              ctypes.c_size_t(flush.numel() * flush.element_size()),
                                              ctypes.byref(us)), "kernel_time")
    return us.value


def launch_count() -> int:
    return int(load().iim_launch_count())


class Engine:
    """Batched engine (see iim.h): admit set-up problems, run ticks, poll, release."""

    def __init__(self, options: Options | None = None, max_slots: int = 64, stream=None):
        import torch
        lib = load()
        self.options = options or default_options()
        self.stream = stream or torch.cuda.current_stream()
        self.max_slots = int(max_slots)
        h = ctypes.c_void_p()
        _check(lib.iim_engine_create(ctypes.byref(self.options), self.max_slots,
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "iim_engine_create")
        self.h = h
        self._done = (ctypes.c_int * self.max_slots)()

    def close(self):
        if getattr(self, "h", None):
            load().iim_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, problem: Problem, x0=None) -> int:
        slot = ctypes.c_int()
        _check(load().iim_engine_admit(self.h, problem.h, _ptr(x0), ctypes.byref(slot)), "iim_engine_admit")
        return slot.value

    def run(self, max_ticks: int = 1 << 30):
        _check(load().iim_engine_run(self.h, int(max_ticks)), "iim_engine_run")

    def poll(self, wait=True):
        """(finished, live, ticks): finished is None while the last run is still on the device."""
        live, nd, ticks = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        st = load().iim_engine_poll(self.h, int(bool(wait)), ctypes.byref(live), self._done, ctypes.byref(nd),
                                    ctypes.byref(ticks))
        if st == IIM_ERR_TIMEOUT and not wait:
            return None, None, None
        _check(st, "iim_engine_poll")
        return [self._done[i] for i in range(nd.value)], live.value, ticks.value

    def release(self, slot: int, x=None, check=True):
        info = SolveInfo()
        _check(load().iim_engine_release(self.h, int(slot), _ptr(x), ctypes.byref(info)), "iim_engine_release")
        if check and info.status != IIM_OK:
            raise IIMError(info.status, f"slot {slot}: " + load().iim_status_string(info.status).decode())
        return info

    def stats(self):
        k, t = ctypes.c_int64(), ctypes.c_int64()
        _check(load().iim_engine_stats(self.h, ctypes.byref(k), ctypes.byref(t)))
        return k.value, t.value

    def set_shapes(self, shapes=None):
        arr = None if shapes is None else (ctypes.c_int * 6)(*shapes)
        _check(load().iim_engine_set_shapes(self.h, arr), "iim_engine_set_shapes")

    def shapes(self):
        arr = (ctypes.c_int * 6)()
        _check(load().iim_engine_get_shapes(self.h, arr))
        return list(arr)

    def autotune(self, reps=3) -> float:
        ms = ctypes.c_double()
        _check(load().iim_engine_autotune(self.h, int(reps), ctypes.byref(ms)), "iim_engine_autotune")
        return ms.value

    def solve_all(self, max_ticks: int = 1 << 30):
        """Run until every admitted slot has finished; returns the tick count of the run."""
        t0 = self.stats()[1]
        self.run(max_ticks)
        self.poll(wait=True)
        return self.stats()[1] - t0


class Server:
    """Request loop over an engine (see iim.h): submit, step, set data, take."""

    def __init__(self, options: Options | None = None, budget_bytes: int = 1 << 34, max_slots: int = 64,
                 ticks_per_run: int = 4, cap: int = 4096, create_threads: int = 8, mode: int = 0, pooling=False):
        lib = load()
        self.options = options or default_options()
        h = ctypes.c_void_p()
        _check(lib.iim_server_create(ctypes.byref(self.options), ctypes.c_size_t(int(budget_bytes)), int(max_slots),
                                     int(ticks_per_run), int(create_threads), ctypes.byref(h)), "iim_server_create")
        self.h = h
        _check(lib.iim_server_set_mode(self.h, int(mode)), "iim_server_set_mode")
        _check(lib.iim_server_set_pooling(self.h, int(bool(pooling))), "iim_server_set_pooling")
        self.mode = mode
        self.cap = cap
        self._need = (ctypes.c_int64 * cap)()
        self._fin = (ctypes.c_int64 * cap)()
        self.descs = {}

    def close(self):
        if getattr(self, "h", None):
            load().iim_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pool_stats(self):
        """(requests that reused a kept problem, requests created afresh, kept problems freed, kept now)"""
        h, m, e, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(load().iim_server_pool_stats(self.h, ctypes.byref(h), ctypes.byref(m), ctypes.byref(e), ctypes.byref(k)))
        return {"hits": h.value, "misses": m.value, "evicted": e.value, "kept": k.value}

    def submit(self, desc: Desc) -> int:
        rid = ctypes.c_int64()
        _check(load().iim_server_submit(self.h, ctypes.byref(desc), ctypes.byref(rid)), "iim_server_submit")
        self.descs[rid.value] = desc
        return rid.value

    def step(self):
        nn, nf = ctypes.c_int(), ctypes.c_int()
        _check(load().iim_server_step(self.h, self._need, self.cap, ctypes.byref(nn), self._fin, self.cap,
                                      ctypes.byref(nf)), "iim_server_step")
        return [self._need[i] for i in range(nn.value)], [self._fin[i] for i in range(nf.value)]

    def problem(self, rid: int) -> Problem:
        h = load().iim_server_problem(self.h, ctypes.c_int64(rid))
        if not h:
            raise IIMError(1, f"request {rid} is not waiting for data")
        return Problem.view(h, self.descs[rid])

    def data_ready(self, rid: int):
        _check(load().iim_server_data_ready(self.h, ctypes.c_int64(rid)), "iim_server_data_ready")

    def cancel(self, rid: int):
        """End a request without a solution (see iim_server_cancel); take() then reports
        IIM_ERR_TIMEOUT for it."""
        _check(load().iim_server_cancel(self.h, ctypes.c_int64(rid)), "iim_server_cancel")

    def take(self, rid: int):
        """(x on the host, SolveInfo, latency seconds, status) of a finished request."""
        import numpy as np
        d = self.descs.pop(rid)
        x = np.zeros(d.n ** d.dim)
        info, lat = SolveInfo(), ctypes.c_double()
        st = load().iim_server_take(self.h, ctypes.c_int64(rid), ctypes.c_void_p(x.ctypes.data), ctypes.byref(info),
                                    ctypes.byref(lat))
        return x, info, lat.value, st

    def stats(self):
        b, pk, q, r, runs = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        hs = (ctypes.c_double * 3)()
        st = (ctypes.c_int * 8)()
        _check(load().iim_server_stats(self.h, ctypes.byref(b), ctypes.byref(pk), ctypes.byref(q), ctypes.byref(r),
                                       ctypes.byref(runs), hs, st))
        return {"bytes_in_use": b.value, "peak_bytes": pk.value, "queued": q.value, "resident": r.value,
                "runs": runs.value, "host_step_s": hs[0], "host_copy_s": hs[1], "host_create_s": hs[2],
                "states": dict(zip(SERVER_STATES, list(st)))}


SERVER_STATES = ("queued", "creating", "need_data", "ready", "running", "retired", "finished", "failed")


def serve(server: Server, arrivals, set_data, realtime=True, idle_sleep=0.0, timings=None, deadline_s=None,
          progress=None, progress_every_s=5.0, data_threads=0):
    """Drive a server through a stream of requests.

    arrivals: list of (arrival time in seconds from now, Desc, user object), sorted by time;
    set_data(problem_view, user) sets the data of a created request.  Returns
    {request id: (x, info, latency, status, user)} and the wall time.  With realtime=False
    every request is submitted at once.  timings (a dict) receives the caller-side host
    seconds spent in step, set_data and take.  With deadline_s, a TimeoutError naming the
    requests' states is raised when requests are still outstanding after that many
    seconds; progress(elapsed_s, taken, outstanding, server stats) is called every
    progress_every_s seconds.  With data_threads > 0, set_data runs on that many client
    threads (each call touches only its own request's problem) and the loop marks a request
    ready once its call has returned, so the loop keeps admitting and collecting meanwhile;
    an exception raised by set_data is raised here.
    """
    import time
    from concurrent.futures import ThreadPoolExecutor
    workers = ThreadPoolExecutor(data_threads) if data_threads > 0 else None
    busy = {}                     # request id -> its set_data call on a client thread
    t0 = time.perf_counter()
    pending = list(arrivals)
    k = 0
    users, out = {}, {}
    outstanding = 0
    t_step = t_data = t_take = 0.0
    next_note = progress_every_s
    while k < len(pending) or outstanding:
        now = time.perf_counter() - t0
        if progress is not None and now >= next_note:
            progress(now, len(out), outstanding, server.stats())
            next_note = now + progress_every_s
        if deadline_s is not None and now > deadline_s:
            raise TimeoutError(f"serve: {outstanding} requests outstanding after {now:.0f} s "
                               f"({len(out)} taken, {len(pending) - k} not submitted): {server.stats()}")
        while k < len(pending) and (not realtime or pending[k][0] <= now):
            _, desc, user = pending[k]
            rid = server.submit(desc)
            users[rid] = user
            outstanding += 1
            k += 1
        a = time.perf_counter()
        need, fin = server.step()
        b = time.perf_counter()
        for rid in need:
            if workers is None:
                set_data(server.problem(rid), users[rid])
                server.data_ready(rid)
            else:
                busy[rid] = workers.submit(set_data, server.problem(rid), users[rid])
        done = [rid for rid, fu in busy.items() if fu.done()]
        for rid in done:
            busy.pop(rid).result()
            server.data_ready(rid)
        c = time.perf_counter()
        for rid in fin:
            x, info, lat, st = server.take(rid)
            out[rid] = (x, info, lat, st, users.pop(rid))
            outstanding -= 1
        d = time.perf_counter()
        t_step += b - a
        t_data += c - b
        t_take += d - c
        if not need and not fin and not done:
            if idle_sleep:
                time.sleep(idle_sleep)
            elif busy:
                time.sleep(2e-4)          # leave the interpreter to the client threads
    if workers is not None:
        workers.shutdown(wait=True)
    if timings is not None:
        timings.update({"step_s": t_step, "set_data_s": t_data, "take_s": t_take})
    return out, time.perf_counter() - t0
