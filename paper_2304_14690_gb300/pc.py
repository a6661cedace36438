"""Python binding of libpc (include/pc.h): argument marshalling only.

Every step of the pressure-correction sub-step runs inside libpc's CUDA kernels; this module
only converts workloads and torch tensors into the C structures and pointers the ABI takes.
If the library has not been built, importing works but every call raises: there is no
fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpc.so")

BC = {"P": 0, "W": 1, "I": 2, "D": 3}
PRECISION = {"fp64": 0, "mixed": 1, "fp32": 2}
DTYPE = {"f64": 0, "f32": 1}
STATUS = ["ok", "invalid argument", "unsupported", "singular WLS system", "out of device memory",
          "device-memory budget exceeded", "CUDA error", "refinement not converged", "timeout"]


PC_OK, PC_ERR_INVALID_ARG, PC_ERR_UNSUPPORTED, PC_ERR_WLS_SINGULAR = 0, 1, 2, 3
PC_ERR_OUT_OF_MEMORY, PC_ERR_BUDGET, PC_ERR_CUDA = 4, 5, 6


class PcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libpc status {status} ({STATUS[status] if status < len(STATUS) else '?'}): {message}")
        self.status = status


class Obstacle(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int), ("centre", ctypes.c_double * 3), ("radius", ctypes.c_double)]


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("lo", ctypes.c_double * 3),
        ("h", ctypes.c_double * 3),
        ("bc_lo", ctypes.c_int * 3),
        ("bc_hi", ctypes.c_int * 3),
        ("num_nodes", ctypes.c_int64),
        ("node_xyz", ctypes.c_void_p),
        ("node_type", ctypes.c_void_p),
        ("num_obstacles", ctypes.c_int),
        ("obstacles", ctypes.POINTER(Obstacle)),
        ("knn", ctypes.c_int),
        ("wls_eps", ctypes.c_double),
        ("support_factor", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("refine_iters", ctypes.c_int),
        ("gauge", ctypes.c_int),
        ("velocity_dtype", ctypes.c_int),
        ("eigenvalues", ctypes.c_int),
        ("divergence", ctypes.c_int),
        ("grid_type", ctypes.c_int),
        ("refine_tol", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("removed_mean", ctypes.c_double),
        ("source_norm", ctypes.c_double),
        ("residual_norm", ctypes.c_double * 9),
        ("refine_iters_done", ctypes.c_int),
        ("max_div_after", ctypes.c_double),
        ("max_abs_u_star", ctypes.c_double),
        ("gauge_shift", ctypes.c_double),
        ("refine_converged", ctypes.c_int),
    ]

    def as_dict(self):
        n = self.refine_iters_done
        return dict(removed_mean=self.removed_mean, source_norm=self.source_norm,
                    residual_norm=list(self.residual_norm[: n + 1]), refine_iters_done=n,
                    max_div_after=self.max_div_after, max_abs_u_star=self.max_abs_u_star,
                    gauge_shift=self.gauge_shift, refine_converged=bool(self.refine_converged))


class Profile(ctypes.Structure):
    _fields_ = [("phase_ms", ctypes.c_double * 8), ("calls", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong)]


PHASES = ("prep", "transfer", "divergence", "transform", "residual", "gauge", "gradient", "stats")


class IbResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("diff", ctypes.c_double), ("prev", ctypes.c_double)]


class ProjectArgs(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("u_star", ctypes.c_void_p), ("f_ib_in", ctypes.c_void_p),
                ("p_out", ctypes.c_void_p), ("u_out", ctypes.c_void_p), ("f_ib_out", ctypes.c_void_p)]


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("h", ctypes.c_double * 3),
        ("bc_lo", ctypes.c_int * 3),
        ("bc_hi", ctypes.c_int * 3),
        ("grid_type", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("refine_iters", ctypes.c_int),
        ("gauge", ctypes.c_int),
        ("eigenvalues", ctypes.c_int),
        ("refine_tol", ctypes.c_double),
    ]


FUNCTIONS = {
    "pc_grid_plan_create": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.c_int, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "pc_plan_create": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.c_int, ctypes.c_size_t,
                                      ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "pc_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(Stats), ctypes.c_void_p]),
    "pc_plan_set_rhs_mask": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pc_project_ib": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(IbResult), ctypes.c_void_p]),
    "pc_project_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ProjectArgs), ctypes.c_void_p]),
    "pc_solve_poisson": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(Stats), ctypes.c_void_p]),
    "pc_plan_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "pc_plan_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "pc_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pc_plan_clone": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "pc_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pc_set_graphs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pc_solve_poisson_static": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "pc_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Profile)]),
    "pc_plan_set_transform_slots": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pc_plan_get_transform_slots": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_int)]),
    "pc_plan_set_transform_ctas": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pc_plan_get_transform_ctas": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int)]),
    "pc_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pc_batcher_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "pc_batcher_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ProjectArgs), ctypes.c_void_p]),
    "pc_batcher_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pc_momentum_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "pc_momentum_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "pc_momentum_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "pc_momentum_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pc_last_error_message": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libpc.so; raises when it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libpc is not built ({LIB_PATH} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in FUNCTIONS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, stats=None):
    """Raise PcError for a failed call; stats (a filled Stats, nullable) travel with the error,
    e.g. the residual norms of a refinement that did not converge."""
    if status != 0:
        err = PcError(status, load().pc_last_error_message().decode())
        err.stats = stats.as_dict() if stats is not None else None
        raise err


def _ptr(x, shape=None, dtype=None, name="array"):
    """Data pointer of a dense torch tensor or numpy array (None -> NULL). The C ABI takes
    plain pointers to dense C-order arrays, so strided views are rejected."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous (C order)")
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {tuple(shape)}")
        if dtype is not None and x.dtype != dtype:
            raise ValueError(f"{name} has dtype {x.dtype}, expected {dtype}")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name} must be C-contiguous")
    return x.ctypes.data


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


GRID_TYPE = {"cells": 0, "vertices": 1}


def vertex_unknowns(lo, hi, n):
    """Pressure unknowns on a vertex-grid axis of n cells with boundary kinds lo, hi."""
    if lo == "P":
        return n
    neu = lambda c: c in ("W", "I")
    if neu(lo) and neu(hi):
        return n + 1
    if not neu(lo) and not neu(hi):
        return n - 1
    return n


EIGENVALUES = {"fd": 0, "spectral": 1}
DIVERGENCE = {"faces": 0, "wls_direct": 1}


# Refinement defaults: at most 4 sweeps, stopping at ||r|| <= 1e-13 ||s|| or at the residual's
# rounding floor (pc_problem_desc.refine_tol).
REFINE_ITERS = 4
REFINE_TOL = 1e-13


def make_desc(problem, precision="fp64", refine_iters=REFINE_ITERS, gauge=0, velocity_dtype=None,
              node_xyz=None, node_type=None, eigenvalues="fd", div_mode="faces", grid_type="cells",
              refine_tol=REFINE_TOL):
    d = ProblemDesc()
    d.dim = problem.dim
    for a in range(3):
        d.n[a] = int(problem.n[a]) if a < problem.dim else 1
        d.lo[a] = float(problem.lo[a]) if a < problem.dim else 0.0
        d.h[a] = float(problem.h[a]) if a < problem.dim else 1.0
        d.bc_lo[a] = BC[problem.bc_lo[a]] if a < problem.dim else 0
        d.bc_hi[a] = BC[problem.bc_hi[a]] if a < problem.dim else 0
    d.num_nodes = problem.num_nodes
    d.node_xyz = _ptr(node_xyz)
    d.node_type = _ptr(node_type)
    d.num_obstacles = 0
    d.obstacles = None
    d.knn = int(problem.knn)
    d.wls_eps = float(problem.eps)
    d.support_factor = float(problem.support_factor)
    d.beta = float(problem.beta)
    d.precision = PRECISION[precision]
    d.refine_iters = int(refine_iters)
    d.refine_tol = float(refine_tol)
    d.gauge = int(gauge)
    if velocity_dtype is None:
        velocity_dtype = "f32" if problem.u_star.dtype == np.float32 else "f64"
    d.velocity_dtype = DTYPE[velocity_dtype]
    d.eigenvalues = EIGENVALUES[eigenvalues]
    d.divergence = DIVERGENCE[div_mode]
    d.grid_type = GRID_TYPE[grid_type]
    return d


class Plan:
    """A libpc plan for one problem geometry (nodes, grid, boundaries)."""

    def __init__(self, problem, precision="fp64", refine_iters=REFINE_ITERS, gauge=0, device=0,
                 budget_bytes=0, stream=None, eigenvalues="fd", div_mode="faces", grid_type="cells",
                 refine_tol=REFINE_TOL):
        import torch
        lib = load()
        self.problem = problem
        self.precision = precision
        self.device = torch.device("cuda", device)
        self.vdtype = torch.float32 if problem.u_star.dtype == np.float32 else torch.float64
        xyz = torch.as_tensor(np.ascontiguousarray(problem.nodes, dtype=np.float64), device=self.device)
        typ = torch.as_tensor(np.ascontiguousarray(problem.node_type, dtype=np.uint8), device=self.device)
        self._desc = make_desc(problem, precision, refine_iters, gauge,
                               "f32" if self.vdtype == torch.float32 else "f64", xyz, typ, eigenvalues, div_mode,
                               grid_type, refine_tol)
        h = ctypes.c_void_p()
        _check(lib.pc_plan_create(ctypes.byref(self._desc), device, budget_bytes,
                                  _stream_handle(stream), ctypes.byref(h)))
        self.handle = h
        self.dim = problem.dim
        self.N = problem.num_nodes
        if grid_type == "vertices":
            # the pressure unknowns of the vertex grid (p_out, the RHS mask)
            self.shape = tuple(vertex_unknowns(problem.bc_lo[a], problem.bc_hi[a], int(problem.n[a]))
                               for a in range(problem.dim))
        else:
            self.shape = tuple(int(v) for v in problem.n[: problem.dim])

    def close(self):
        if getattr(self, "handle", None):
            _check(load().pc_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clone(self, stream=None):
        """pc_plan_clone: another workspace on the same rows and tables (the clone keeps its
        root alive)."""
        h = ctypes.c_void_p()
        _check(load().pc_plan_clone(self.handle, _stream_handle(stream), ctypes.byref(h)))
        c = Plan.__new__(Plan)
        c.__dict__.update({k: v for k, v in self.__dict__.items() if k != "handle"})
        c._root = getattr(self, "_root", None) or self
        c.handle = h
        return c

    def nbytes(self):
        b = ctypes.c_size_t()
        _check(load().pc_plan_bytes(self.handle, ctypes.byref(b)))
        return b.value

    def graphs(self, on=True):
        _check(load().pc_set_graphs(self.handle, 1 if on else 0))

    def _prec_code(self, precision):
        return PRECISION[precision if precision is not None else self.precision]

    def set_slots(self, axis, slots, precision=None):
        """Slots per thread of the transform passes along axis (2, 4, 8 or 16; for FP32 passes
        also 0 and 1: variant 0 or 1 of the compile-time pass of the axis length where it has
        one; 0 is the default)."""
        _check(load().pc_plan_set_transform_slots(self.handle, axis, self._prec_code(precision), slots))

    def slots(self, precision=None):
        """Current slots per thread of every axis for the given (default: the plan's) precision."""
        out = []
        for a in range(self.dim):
            v = ctypes.c_int()
            _check(load().pc_plan_get_transform_slots(self.handle, a, self._prec_code(precision), ctypes.byref(v)))
            out.append(v.value)
        return out

    def set_ctas(self, axis, ctas_per_sm, precision=None):
        """CTAs per SM the single-problem passes along axis aim for (1, 2, 4 or 8)."""
        _check(load().pc_plan_set_transform_ctas(self.handle, axis, self._prec_code(precision), ctas_per_sm))

    def ctas(self, precision=None):
        """Current CTA target of every axis for the given (default: the plan's) precision."""
        out = []
        for a in range(self.dim):
            v = ctypes.c_int()
            _check(load().pc_plan_get_transform_ctas(self.handle, a, self._prec_code(precision), ctypes.byref(v)))
            out.append(v.value)
        return out

    def autotune(self, stream=None):
        """Time the plan's transform solve for every slot count and CTA target of every axis
        and keep the fastest schedule; returns its milliseconds per solve."""
        ms = ctypes.c_double()
        _check(load().pc_plan_autotune(self.handle, _stream_handle(stream), ctypes.byref(ms)))
        return ms.value

    def profile(self, on=True):
        _check(load().pc_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self):
        """Per-phase milliseconds summed over the calls since the last read, calls, launches."""
        pr = Profile()
        _check(load().pc_profile_read(self.handle, ctypes.byref(pr)))
        return dict(phase_ms={PHASES[i]: pr.phase_ms[i] for i in range(8)}, calls=pr.calls,
                    kernel_launches=pr.kernel_launches)

    def rows(self, which):
        """(col [rows, K] int32, w) of face axis `which` (w [rows, K]), of the nodes
        (which == dim, w [dim, rows, K]) or of the cell centres of a direct-divergence plan
        (which == dim + 1, w [dim, rows, K])."""
        lib = load()
        n = ctypes.c_int64()
        _check(lib.pc_plan_rows(self.handle, which, ctypes.byref(n), None, None))
        K = 3 ** self.dim if which == self.dim else self.problem.knn
        nw = 1 if which < self.dim else self.dim
        col = np.empty((n.value, K), dtype=np.int32)
        w = np.empty((nw, n.value, K), dtype=np.float64)
        _check(lib.pc_plan_rows(self.handle, which, ctypes.byref(n), col.ctypes.data, w.ctypes.data))
        return col, (w if which >= self.dim else w[0])

    def alloc_outputs(self):
        import torch
        p = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        u = torch.empty((self.dim, self.N), dtype=self.vdtype, device=self.device)
        f = torch.empty((self.dim, self.N), dtype=self.vdtype, device=self.device)
        return p, u, f

    def project(self, u_star, f_ib=None, dt=None, out=None, stats=False, stream=None):
        """Run pc_project. u_star/f_ib: torch tensors (device or host) [dim, N].
        Returns (p, u_out, f_out, stats_dict or None)."""
        lib = load()
        if dt is None:
            dt = self.problem.dt
        p, u, f = out if out is not None else self.alloc_outputs()
        st = Stats() if stats else None
        vshape = (self.dim, self.N)
        _check(lib.pc_project(self.handle, float(dt), _ptr(u_star, vshape, self.vdtype, "u_star"),
                              _ptr(f_ib, vshape, self.vdtype, "f_ib"),
                              _ptr(p, self.shape, None, "p_out"), _ptr(u, vshape, self.vdtype, "u_out"),
                              _ptr(f, vshape, self.vdtype, "f_out"),
                              ctypes.byref(st) if st is not None else None, _stream_handle(stream)), st)
        return p, u, f, (st.as_dict() if st is not None else None)

    def set_rhs_mask(self, mask, stream=None):
        """pc_plan_set_rhs_mask: mask (cells, uint8, nonzero = flow domain; numpy array or
        torch tensor) or None to clear."""
        import torch
        if mask is not None and not hasattr(mask, "data_ptr"):
            mask = torch.as_tensor(np.ascontiguousarray(mask, dtype=np.uint8))
        _check(load().pc_plan_set_rhs_mask(self.handle, _ptr(mask, self.shape, torch.uint8, "mask"),
                                           _stream_handle(stream)))

    def project_ib(self, u_star, f_init=None, tol=1e-3, max_iters=50, dt=None, out=None, stream=None):
        """Run pc_project_ib (the IB-force iteration) on device tensors [dim, N].
        Returns (p, u_out, f_out, info) with info = dict(iterations, converged, diff, prev,
        history=[(diff, prev) per pass])."""
        lib = load()
        if dt is None:
            dt = self.problem.dt
        p, u, f = out if out is not None else self.alloc_outputs()
        vshape = (self.dim, self.N)
        hist = (ctypes.c_double * (2 * int(max_iters)))()
        res = IbResult()
        _check(lib.pc_project_ib(self.handle, float(dt), _ptr(u_star, vshape, self.vdtype, "u_star"),
                                 _ptr(f_init, vshape, self.vdtype, "f_init"), float(tol), int(max_iters),
                                 _ptr(p, self.shape, None, "p_out"), _ptr(u, vshape, self.vdtype, "u_out"),
                                 _ptr(f, vshape, self.vdtype, "f_out"), hist, ctypes.byref(res),
                                 _stream_handle(stream)))
        n = res.iterations
        info = dict(iterations=n, converged=bool(res.converged), diff=res.diff, prev=res.prev,
                    history=[(hist[2 * k], hist[2 * k + 1]) for k in range(n)])
        return p, u, f, info

    def solve_poisson(self, s, p_out=None, stats=False, stream=None):
        import torch
        lib = load()
        if p_out is None:
            p_out = torch.empty(self.shape, dtype=torch.float64, device=s.device)
        st = Stats() if stats else None
        _check(lib.pc_solve_poisson(self.handle, _ptr(s, self.shape, torch.float64, "s"),
                                    _ptr(p_out, self.shape, torch.float64, "p_out"),
                                    ctypes.byref(st) if st is not None else None, _stream_handle(stream)), st)
        return p_out, (st.as_dict() if st is not None else None)


class GridPlan(Plan):
    """A grid-only plan (pc_grid_plan_create): the Poisson solve alone, on the cell-centred or
    the vertex pressure grid. solve_poisson, autotune and the schedule controls apply; the node
    entry points do not."""

    def __init__(self, dim, n, h, bc_lo, bc_hi, grid_type="cells", precision="fp64", refine_iters=REFINE_ITERS,
                 gauge=0, eigenvalues="fd", device=0, stream=None, refine_tol=REFINE_TOL):
        import torch
        lib = load()
        d = GridDesc()
        d.dim = dim
        for a in range(3):
            d.n[a] = int(n[a]) if a < dim else 1
            d.h[a] = float(h[a]) if a < dim else 1.0
            d.bc_lo[a] = BC[bc_lo[a]] if a < dim else 0
            d.bc_hi[a] = BC[bc_hi[a]] if a < dim else 0
        d.grid_type = GRID_TYPE[grid_type]
        d.precision = PRECISION[precision]
        d.refine_iters = int(refine_iters)
        d.refine_tol = float(refine_tol)
        d.gauge = int(gauge)
        d.eigenvalues = EIGENVALUES[eigenvalues]
        self._gdesc = d
        self.precision = precision
        self.device = torch.device("cuda", device)
        self.dim = dim
        self.N = 0
        h_ = ctypes.c_void_p()
        _check(lib.pc_grid_plan_create(ctypes.byref(d), device, _stream_handle(stream), ctypes.byref(h_)))
        self.handle = h_
        if grid_type == "vertices":
            self.shape = tuple(vertex_unknowns(bc_lo[a], bc_hi[a], int(n[a])) for a in range(dim))
        else:
            self.shape = tuple(int(n[a]) for a in range(dim))


class Momentum:
    """pc_momentum: the AB2 predictor of Eq. 3 on a plan's nodes. predict(u_n, dt) returns u*;
    correct it with the plan (project / project_ib, same dt) and feed the corrected velocity to
    the next predict."""

    def __init__(self, plan, nu=0.0, force=None, knn=None, stream=None):
        lib = load()
        self.plan = plan
        prob = plan.problem
        xyz = np.ascontiguousarray(prob.nodes, dtype=np.float64)
        f = None
        if force is not None:
            f = (ctypes.c_double * 3)(*[float(force[a]) if a < plan.dim else 0.0 for a in range(3)])
        h = ctypes.c_void_p()
        _check(lib.pc_momentum_create(plan.handle, xyz.ctypes.data, int(knn or prob.knn), float(nu), f,
                                      _stream_handle(stream), ctypes.byref(h)))
        self.handle = h
        self._shape = (plan.dim, plan.N)
        self._dtype = plan.vdtype
        self._device = plan.device

    def predict(self, u_n, dt, u_boundary=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self._shape, dtype=self._dtype, device=self._device)
        _check(load().pc_momentum_predict(self.handle, float(dt), _ptr(u_n, self._shape, self._dtype, "u_n"),
                                          _ptr(u_boundary, self._shape, self._dtype, "u_boundary"),
                                          _ptr(out, self._shape, self._dtype, "u_star"), _stream_handle(stream)))
        return out

    def reset(self):
        _check(load().pc_momentum_reset(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            _check(load().pc_momentum_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_poisson_static(dim, n, h, bc_lo, bc_hi, s, p_out, gauge=0, stream=None):
    """pc_solve_poisson_static: allocation-free FP64 Poisson solve on device tensors."""
    import torch
    lib = load()
    shape = tuple(int(v) for v in n[:dim])
    nn = (ctypes.c_int64 * 3)(*[int(n[a]) if a < dim else 1 for a in range(3)])
    hh = (ctypes.c_double * 3)(*[float(h[a]) if a < dim else 1.0 for a in range(3)])
    lo = (ctypes.c_int * 3)(*[BC[bc_lo[a]] if a < dim else 0 for a in range(3)])
    hi = (ctypes.c_int * 3)(*[BC[bc_hi[a]] if a < dim else 0 for a in range(3)])
    _check(lib.pc_solve_poisson_static(dim, nn, hh, lo, hi, int(gauge),
                                       _ptr(s, shape, torch.float64, "s"),
                                       _ptr(p_out, shape, torch.float64, "p_out"), _stream_handle(stream)))
    return p_out


def _batch_arrays(plans, args):
    n = len(plans)
    hs = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    arr = (ProjectArgs * n)()
    for i, a in enumerate(args):
        arr[i].dt = float(a["dt"])
        arr[i].u_star = _ptr(a["u_star"])
        arr[i].f_ib_in = _ptr(a.get("f_ib"))
        arr[i].p_out = _ptr(a["p"])
        arr[i].u_out = _ptr(a["u"])
        arr[i].f_ib_out = _ptr(a.get("f"))
    return n, hs, arr


def project_batch(plans, args, stream=None):
    """pc_project_batch over (plan, dict(dt, u_star, f_ib, p, u, f)) pairs (device tensors)."""
    n, hs, arr = _batch_arrays(plans, args)
    _check(load().pc_project_batch(n, hs, arr, _stream_handle(stream)))


class Batcher:
    """pc_batcher: launches batches that change from call to call, without capture or
    allocation per call (see include/pc.h)."""

    def __init__(self, device=0, table_bytes=0, slots=4):
        h = ctypes.c_void_p()
        _check(load().pc_batcher_create(device, table_bytes, slots, ctypes.byref(h)))
        self.handle = h

    def launch(self, plans, args, stream=None):
        n, hs, arr = _batch_arrays(plans, args)
        _check(load().pc_batcher_launch(self.handle, n, hs, arr, _stream_handle(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().pc_batcher_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
