"""Thin ctypes binding of libibdl (argument marshalling only).

Every computation happens in the CUDA library; this module converts torch
tensors or numpy arrays to raw pointers, fills the C structs of
``include/ibdl.h`` and turns error codes into exceptions.  The names follow
the C entry points: ``create_geometry``, ``apply``, ``solve``, ``evaluate``,
``spread_div``, ``spread``, ``helmholtz``, ``interp``.

Arrays may live on the GPU (torch CUDA tensors) or on the host (numpy arrays
or CPU tensors, pinned or not); the library copies host arrays itself.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibdl.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
ERR_BREAKDOWN, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = 5, 6, 7, 8
DIRICHLET, NEUMANN = 0, 1
DELTA = {"peskin4": 0, "cos4": 1}
FP64, FP32_REFINED = 0, 1
DISC = {"fd": 0, "spectral": 1}

# Every function that include/ibdl.h declares (the ABI test checks this list
# against the header and the library's exports).
EXPORTS = [
    "ibdl_solve_opts_default", "ibdl_create_geometry", "ibdl_destroy_geometry",
    "ibdl_apply", "ibdl_apply_precision", "ibdl_solve", "ibdl_evaluate",
    "ibdl_spread_div", "ibdl_spread", "ibdl_helmholtz", "ibdl_interp",
    "ibdl_get_geometry_info", "ibdl_kernel_launch_count", "ibdl_profile_enable",
    "ibdl_profile_read", "ibdl_status_string",
    "ibdl_last_error_message", "ibdl_version", "ibdl_helmholtz_2d_noalloc",
    "ibdl_batch_create", "ibdl_batch_destroy", "ibdl_solve_batched",
    "ibdl_server_config_default", "ibdl_server_create", "ibdl_server_destroy",
    "ibdl_server_clock", "ibdl_server_submit", "ibdl_server_step", "ibdl_server_take",
    "ibdl_server_get_stats", "ibdl_tuning_enable", "ibdl_tuning_set", "ibdl_indicator",
    "ibdl_near_boundary", "ibdl_selftest_bounded_wait", "ibdl_solver_smem_query",
    "ibdl_tuning_set_pencils", "ibdl_profile_trace", "ibdl_profile_trace_read",
    "ibdl_geometry_set_solver_pencils", "ibdl_tuning_set_plan",
]


class GeometryDesc(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("n", C.c_int32), ("box_len", C.c_double),
        ("origin", C.c_double * 3), ("m", C.c_int64),
        ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
        ("nx", C.c_void_p), ("ny", C.c_void_p), ("nz", C.c_void_p),
        ("w", C.c_void_p), ("kappa", C.c_double), ("delta", C.c_int32),
        ("bc", C.c_int32), ("precision", C.c_int32), ("disc", C.c_int32),
        ("eta", C.c_double),
    ]


class SolveOpts(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("restart", C.c_int32), ("max_iters", C.c_int32),
        ("max_refine", C.c_int32), ("engine", C.c_int32), ("inner_tol", C.c_double),
        ("x0", C.c_void_p),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int32), ("refine_steps", C.c_int32), ("matvecs", C.c_int32),
        ("n_history", C.c_int32), ("rel_residual", C.c_double),
        ("residual_history", C.c_double * 256), ("residual_updates", C.c_int32),
    ]

    def as_dict(self):
        return {"iters": self.iters, "refine_steps": self.refine_steps,
                "matvecs": self.matvecs, "rel_residual": self.rel_residual,
                "residual_updates": self.residual_updates,
                "history": list(self.residual_history[: self.n_history])}


class GeometryInfo(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("n", C.c_int32), ("m", C.c_int64), ("h", C.c_double),
        ("kappa", C.c_double), ("bc", C.c_int32), ("delta", C.c_int32),
        ("precision", C.c_int32), ("device_bytes", C.c_int64),
        ("fft_passes", C.c_int32), ("rows_per_tile", C.c_int32),
        ("pencils_per_item", C.c_int32 * 2), ("fft_plan", C.c_int32),
    ]


class ServerConfig(C.Structure):
    _fields_ = [
        ("memory_budget", C.c_int64), ("max_active", C.c_int32),
        ("rounds_per_step", C.c_int32), ("reserve_sms", C.c_int32), ("reserved", C.c_int32),
        ("opts", SolveOpts),
    ]


class RequestResult(C.Structure):
    _fields_ = [
        ("id", C.c_int64), ("status", C.c_int32), ("slot", C.c_int32),
        ("t_arrival", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
        ("device_bytes", C.c_int64), ("info", SolveInfo),
    ]


class ServerStats(C.Structure):
    _fields_ = [
        ("queued", C.c_int32), ("active", C.c_int32), ("finished", C.c_int32),
        ("reserved", C.c_int32), ("bytes_in_use", C.c_int64), ("peak_bytes", C.c_int64),
        ("memory_budget", C.c_int64), ("steps", C.c_int64), ("launches", C.c_int64),
        ("submitted", C.c_int64), ("admit_seconds", C.c_double), ("wait_seconds", C.c_double),
    ]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double)]


class IbdlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ibdl status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libibdl.so (built by ``build.py``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libibdl.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "ibdl_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
        "ibdl_create_geometry": (C.c_int, [C.POINTER(GeometryDesc), vp, C.POINTER(vp)]),
        "ibdl_destroy_geometry": (None, [vp]),
        "ibdl_apply": (C.c_int, [vp, vp, vp, vp]),
        "ibdl_apply_precision": (C.c_int, [vp, vp, vp, i32, vp]),
        "ibdl_solve": (C.c_int, [vp, vp, vp, vp, C.POINTER(SolveOpts),
                                 C.POINTER(SolveInfo), vp]),
        "ibdl_evaluate": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "ibdl_spread_div": (C.c_int, [vp, vp, vp, i32, vp]),
        "ibdl_spread": (C.c_int, [vp, vp, vp, i32, vp]),
        "ibdl_helmholtz": (C.c_int, [vp, vp, vp, i32, vp]),
        "ibdl_interp": (C.c_int, [vp, vp, vp, i32, vp]),
        "ibdl_get_geometry_info": (C.c_int, [vp, C.POINTER(GeometryInfo)]),
        "ibdl_kernel_launch_count": (i64, []),
        "ibdl_profile_enable": (None, [i32]),
        "ibdl_profile_read": (i32, [C.POINTER(KernelStat), i32, i32]),
        "ibdl_status_string": (C.c_char_p, [C.c_int]),
        "ibdl_last_error_message": (C.c_char_p, []),
        "ibdl_version": (i32, []),
        "ibdl_helmholtz_2d_noalloc": (C.c_int, [i32, C.c_double, C.c_double, vp, vp, vp]),
        "ibdl_batch_create": (C.c_int, [i32, C.POINTER(vp)]),
        "ibdl_batch_destroy": (None, [vp]),
        "ibdl_solve_batched": (C.c_int, [vp, i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                         C.POINTER(SolveOpts), C.POINTER(SolveInfo),
                                         C.POINTER(C.c_int), vp]),
        "ibdl_server_config_default": (None, [C.POINTER(ServerConfig)]),
        "ibdl_server_create": (C.c_int, [C.POINTER(ServerConfig), C.POINTER(vp)]),
        "ibdl_server_destroy": (None, [vp]),
        "ibdl_server_clock": (C.c_double, []),
        "ibdl_server_submit": (C.c_int, [vp, C.POINTER(GeometryDesc), vp, C.c_double,
                                         C.POINTER(i64)]),
        "ibdl_server_step": (C.c_int, [vp, C.POINTER(i64), i32, C.POINTER(i32)]),
        "ibdl_server_take": (C.c_int, [vp, i64, vp, C.POINTER(RequestResult)]),
        "ibdl_server_get_stats": (C.c_int, [vp, C.POINTER(ServerStats)]),
        "ibdl_tuning_enable": (None, [i32]),
        "ibdl_tuning_set": (i32, [i32, i32, i32, i32]),
        "ibdl_indicator": (C.c_int, [vp, vp, vp, vp]),
        "ibdl_near_boundary": (C.c_int, [vp, vp, vp, vp, i32, C.c_double, vp, vp]),
        "ibdl_selftest_bounded_wait": (C.c_int, [C.c_uint32, vp]),
        "ibdl_solver_smem_query": (C.c_int, [i32, i32, i32, i32, C.POINTER(i64),
                                             C.POINTER(i64), C.POINTER(i32)]),
        "ibdl_tuning_set_pencils": (C.c_int, [i32, i32, i32, i32, i32]),
        "ibdl_tuning_set_plan": (C.c_int, [i32, i32, i32, i32]),
        "ibdl_profile_trace": (C.c_int, [i32]),
        "ibdl_profile_trace_read": (i64, [vp, i64]),
        "ibdl_geometry_set_solver_pencils": (C.c_int, [vp, i32, i32, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != OK:
        lib = load()
        raise IbdlError(status, lib.ibdl_status_string(status).decode() + ": "
                        + lib.ibdl_last_error_message().decode())


def _ptr(a):
    """Raw address of a contiguous float64 tensor / array (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("numpy arrays must be contiguous float64")
        return a.ctypes.data
    # torch tensor
    if str(a.dtype) != "torch.float64" or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    return a.data_ptr()


def _ptr_u8(a):
    """Raw address of a contiguous uint8 tensor / array (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.uint8 or not a.flags.c_contiguous:
            raise TypeError("masks must be contiguous uint8 arrays")
        return a.ctypes.data
    if str(a.dtype) != "torch.uint8" or not a.is_contiguous():
        raise TypeError("masks must be contiguous uint8 tensors")
    return a.data_ptr()


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def kernel_launch_count() -> int:
    return int(load().ibdl_kernel_launch_count())


def profile_enable(on: bool = True) -> None:
    """Bracket every library launch with CUDA events (see ibdl.h)."""
    load().ibdl_profile_enable(1 if on else 0)


def profile_read(reset: bool = True) -> dict:
    """{kernel family: (launches, total_ms)} from the library's event pairs."""
    lib = load()
    k = lib.ibdl_profile_read(None, 0, 0)
    arr = (KernelStat * max(k, 1))()
    k = lib.ibdl_profile_read(arr, k, 1 if reset else 0)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(k)}


def profile_trace(on: bool = True) -> None:
    """Switch the persistent solver's work-item trace on or off (profiling
    must be on)."""
    _check(load().ibdl_profile_trace(1 if on else 0))


TRACE_CAP = 1 << 16


def profile_trace_read():
    """(records, count): the trace records as a (k, 3) uint64 array (start
    ns, end ns, packed ids; see ibdl.h) and their number; clears the trace."""
    import numpy as np
    out = np.zeros((TRACE_CAP, 3), dtype=np.uint64)
    k = int(load().ibdl_profile_trace_read(out.ctypes.data, TRACE_CAP))
    if k < 0:
        raise IbdlError(ERR_CUDA, "trace read failed")
    return out[:k].copy(), k


def selftest_bounded_wait(spin_limit=1 << 16, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status (TIMEOUT expected)."""
    return int(load().ibdl_selftest_bounded_wait(int(spin_limit), _stream(stream)))


def helmholtz_2d_noalloc(n, box_len, kappa, f, v_out, stream=None):
    """v_out = kappa L'^{-1} f on an n x n periodic grid without any device
    allocation (for callers that cannot allocate; device arrays only, n <= 512;
    overlapping calls race on the library's shared scratch)."""
    _check(load().ibdl_helmholtz_2d_noalloc(int(n), float(box_len), float(kappa), _ptr(f),
                                            _ptr(v_out), _stream(stream)))
    return v_out


def solver_smem_query(dim: int, n: int, rows: int, elem: int) -> dict:
    """Shared memory of one solver work item per kind for element type elem
    (0 float64, 1 float32, 2 double-float), the launch's reservation and the
    twiddle-table length (host only; see ibdl.h)."""
    need = (C.c_int64 * 3)()
    budget, ntw = C.c_int64(), C.c_int32()
    _check(load().ibdl_solver_smem_query(int(dim), int(n), int(rows), int(elem), need,
                                         C.byref(budget), C.byref(ntw)))
    return {"need": [int(v) for v in need], "budget": int(budget.value),
            "twiddles": int(ntw.value)}


def tuning_enable(on: bool = True) -> None:
    load().ibdl_tuning_enable(1 if on else 0)


def tuning_set(dim: int, n: int, precision: int, rows: int) -> None:
    """Pin the x-pass tiling of (current device, dim, n, precision); rows = 0
    drops the pin."""
    _check(load().ibdl_tuning_set(int(dim), int(n), int(precision), int(rows)))


def tuning_set_pencils(dim: int, n: int, precision: int, c_solve: int, c_y: int = 0) -> None:
    """Pin the pencils per work item of (current device, dim, n, precision);
    both 0 drops the pin."""
    _check(load().ibdl_tuning_set_pencils(int(dim), int(n), int(precision), int(c_solve),
                                          int(c_y)))


def tuning_set_plan(dim: int, n: int, precision: int, plan: int) -> None:
    """Pin the float32 FFT plan variant of (current device, dim, n,
    precision); -1 drops the pin."""
    _check(load().ibdl_tuning_set_plan(int(dim), int(n), int(precision), int(plan)))


def version() -> int:
    return int(load().ibdl_version())


def make_desc(dim, n, box_len, origin, x, y, nx, ny, w, kappa, z=None, nz=None,
              delta="peskin4", bc=DIRICHLET, precision=FP64, eta=0.0, disc=0):
    """Fill an ``ibdl_geometry_desc`` (the arrays must outlive its use)."""
    d = GeometryDesc()
    d.dim, d.n, d.box_len = int(dim), int(n), float(box_len)
    org = list(origin) + [0.0] * (3 - len(origin))
    d.origin = (C.c_double * 3)(*org[:3])
    d.m = int(len(x))
    d.x, d.y, d.z = _ptr(x), _ptr(y), _ptr(z)
    d.nx, d.ny, d.nz = _ptr(nx), _ptr(ny), _ptr(nz)
    d.w = _ptr(w)
    d.kappa = float(kappa)
    d.delta = DELTA[delta] if isinstance(delta, str) else int(delta)
    d.bc, d.precision = int(bc), int(precision)
    d.eta = float(eta)
    d.disc = DISC[disc] if isinstance(disc, str) else int(disc)
    return d


def workload_arrays(geom):
    """Contiguous float64 columns (x, y, z, nx, ny, nz, w) of a workload geometry."""
    X = np.ascontiguousarray(geom.X, dtype=np.float64)
    N = np.ascontiguousarray(geom.normals, dtype=np.float64)
    cols = [np.ascontiguousarray(X[:, c]) for c in range(geom.dim)]
    ncols = [np.ascontiguousarray(N[:, c]) for c in range(geom.dim)]
    z = cols[2] if geom.dim == 3 else None
    nz = ncols[2] if geom.dim == 3 else None
    return (cols[0], cols[1], z, ncols[0], ncols[1], nz,
            np.ascontiguousarray(geom.weights, dtype=np.float64))


class Server:
    """Continuous-batching solve server (``ibdl_server_*``)."""

    def __init__(self, memory_budget=0, max_active=64, rounds_per_step=8, reserve_sms=8,
                 tol=1e-8, restart=30, max_iters=500, max_refine=8, inner_tol=1e-5):
        lib = load()
        cfg = ServerConfig()
        lib.ibdl_server_config_default(C.byref(cfg))
        cfg.memory_budget, cfg.max_active = int(memory_budget), int(max_active)
        cfg.rounds_per_step, cfg.reserve_sms = int(rounds_per_step), int(reserve_sms)
        cfg.opts.tol, cfg.opts.restart = float(tol), int(restart)
        cfg.opts.max_iters, cfg.opts.max_refine = int(max_iters), int(max_refine)
        cfg.opts.inner_tol = float(inner_tol)
        h = C.c_void_p()
        _check(lib.ibdl_server_create(C.byref(cfg), C.byref(h)))
        self._h = h

    @staticmethod
    def clock():
        return float(load().ibdl_server_clock())

    def submit(self, geom, bdata, bc=DIRICHLET, precision=FP32_REFINED, t_arrival=-1.0):
        """Queue a workload geometry with its boundary data; returns the request id."""
        x, y, z, nx, ny, nz, w = workload_arrays(geom)
        d = make_desc(geom.dim, geom.n, geom.box_len, geom.origin, x, y, nx, ny, w,
                      geom.kappa, z=z, nz=nz, delta=geom.delta, bc=bc, precision=precision)
        b = np.ascontiguousarray(bdata, dtype=np.float64)
        rid = C.c_int64()
        _check(load().ibdl_server_submit(self._h, C.byref(d), _ptr(b), float(t_arrival),
                                         C.byref(rid)))
        return int(rid.value)

    def step(self, max_ids=4096):
        """One scheduling step; returns the ids finished in it."""
        ids = (C.c_int64 * max_ids)()
        nd = C.c_int32()
        _check(load().ibdl_server_step(self._h, ids, int(max_ids), C.byref(nd)))
        return [int(ids[i]) for i in range(min(nd.value, max_ids))]

    def take(self, rid, m):
        """(q, record) of a finished request."""
        q = np.empty(int(m), dtype=np.float64)
        r = RequestResult()
        _check(load().ibdl_server_take(self._h, int(rid), _ptr(q), C.byref(r)))
        rec = {"id": r.id, "status": r.status, "slot": r.slot, "t_arrival": r.t_arrival,
               "t_admit": r.t_admit, "t_done": r.t_done, "device_bytes": r.device_bytes}
        rec.update(r.info.as_dict())
        return q, rec

    def stats(self):
        s = ServerStats()
        _check(load().ibdl_server_get_stats(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            load().ibdl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    """An IBDL problem's geometry handle (``ibdl_create_geometry``).

    ``x, y, z, nx, ny, nz, w`` are float64 arrays of length m (host or
    device); they are copied by the library.
    """

    def __init__(self, dim, n, box_len, origin, x, y, nx, ny, w, kappa, z=None,
                 nz=None, delta="peskin4", bc=DIRICHLET, precision=FP64, stream=None,
                 eta=0.0, disc=0):
        lib = load()
        d = GeometryDesc()
        d.dim, d.n, d.box_len = int(dim), int(n), float(box_len)
        org = list(origin) + [0.0] * (3 - len(origin))
        d.origin = (C.c_double * 3)(*org[:3])
        d.m = int(len(x))
        d.x, d.y, d.z = _ptr(x), _ptr(y), _ptr(z)
        d.nx, d.ny, d.nz = _ptr(nx), _ptr(ny), _ptr(nz)
        d.w = _ptr(w)
        d.kappa = float(kappa)
        d.delta = DELTA[delta] if isinstance(delta, str) else int(delta)
        d.bc, d.precision = int(bc), int(precision)
        d.eta = float(eta)
        d.disc = DISC[disc] if isinstance(disc, str) else int(disc)
        self._keep = (x, y, z, nx, ny, nz, w)
        h = C.c_void_p()
        _check(lib.ibdl_create_geometry(C.byref(d), _stream(stream), C.byref(h)))
        self._h = h
        self._keep = None
        self.dim, self.n, self.m = d.dim, d.n, d.m
        self.bc, self.precision = d.bc, d.precision
        self.eta = d.eta
        self.nsys = d.m + 1 if d.eta > 0 else d.m

    @classmethod
    def from_workload(cls, geom, bc=DIRICHLET, precision=FP64, stream=None, eta=0.0,
                      disc=0):
        """Build from a ``workloads.geometry.Geometry`` (host float64)."""
        X = np.ascontiguousarray(geom.X, dtype=np.float64)
        N = np.ascontiguousarray(geom.normals, dtype=np.float64)
        cols = [np.ascontiguousarray(X[:, c]) for c in range(geom.dim)]
        ncols = [np.ascontiguousarray(N[:, c]) for c in range(geom.dim)]
        return cls(geom.dim, geom.n, geom.box_len, geom.origin, cols[0], cols[1], ncols[0],
                   ncols[1], np.ascontiguousarray(geom.weights, dtype=np.float64),
                   geom.kappa, z=cols[2] if geom.dim == 3 else None,
                   nz=ncols[2] if geom.dim == 3 else None, delta=geom.delta, bc=bc,
                   precision=precision, stream=stream, eta=eta, disc=disc)

    def close(self):
        if getattr(self, "_h", None):
            load().ibdl_destroy_geometry(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        gi = GeometryInfo()
        _check(load().ibdl_get_geometry_info(self._h, C.byref(gi)))
        out = {}
        for f, _ in GeometryInfo._fields_:
            v = getattr(gi, f)
            out[f] = list(v) if isinstance(v, C.Array) else v
        return out

    def set_solver_pencils(self, c_f64=0, c_f32=0, c_dd=0):
        """Pencils per work item of the persistent solver's solve pass, per
        element type (0: the fixed rule)."""
        _check(load().ibdl_geometry_set_solver_pencils(self._h, int(c_f64), int(c_f32),
                                                       int(c_dd)))

    def apply(self, q, y, precision=None, stream=None):
        lib = load()
        if precision is None:
            _check(lib.ibdl_apply(self._h, _ptr(q), _ptr(y), _stream(stream)))
        else:
            _check(lib.ibdl_apply_precision(self._h, _ptr(q), _ptr(y), int(precision),
                                            _stream(stream)))
        return y

    def solve(self, bdata, q_out, g_grid=None, tol=1e-8, restart=30, max_iters=500,
              max_refine=8, inner_tol=1e-5, x0=None, stream=None, raise_on_error=True,
              engine=0):
        o = SolveOpts()
        load().ibdl_solve_opts_default(C.byref(o))
        o.tol, o.restart, o.max_iters = float(tol), int(restart), int(max_iters)
        o.max_refine, o.inner_tol, o.x0 = int(max_refine), float(inner_tol), _ptr(x0)
        o.engine = int(engine)
        info = SolveInfo()
        st = load().ibdl_solve(self._h, _ptr(bdata), _ptr(g_grid), _ptr(q_out), C.byref(o),
                               C.byref(info), _stream(stream))
        if raise_on_error:
            _check(st)
        out = info.as_dict()
        out["status"] = int(st)
        return out

    def evaluate(self, q, u_out, vb=None, g_grid=None, stream=None):
        _check(load().ibdl_evaluate(self._h, _ptr(q), _ptr(vb), _ptr(g_grid), _ptr(u_out),
                                    _stream(stream)))
        return u_out

    def indicator(self, chi_h_out=None, chi_out=None, stream=None):
        """App. D indicator: chi_h (float64 grid) and chi (uint8 grid)."""
        _check(load().ibdl_indicator(self._h, _ptr(chi_h_out), _ptr_u8(chi_out),
                                     _stream(stream)))
        return chi_h_out, chi_out

    def near_boundary(self, u_in, ub, inside, m1, m2, u_out, stream=None):
        """App. A near-boundary values (2D): u_out from u_in."""
        _check(load().ibdl_near_boundary(self._h, _ptr(u_in), _ptr(ub), _ptr_u8(inside),
                                         int(m1), float(m2), _ptr(u_out), _stream(stream)))
        return u_out

    def spread_div(self, q, f_out, precision=FP64, stream=None):
        _check(load().ibdl_spread_div(self._h, _ptr(q), _ptr(f_out), int(precision),
                                      _stream(stream)))
        return f_out

    def spread(self, v, f_out, precision=FP64, stream=None):
        _check(load().ibdl_spread(self._h, _ptr(v), _ptr(f_out), int(precision),
                                  _stream(stream)))
        return f_out

    def helmholtz(self, f, v_out, precision=FP64, stream=None):
        _check(load().ibdl_helmholtz(self._h, _ptr(f), _ptr(v_out), int(precision),
                                     _stream(stream)))
        return v_out

    def interp(self, u, y_out, precision=FP64, stream=None):
        _check(load().ibdl_interp(self._h, _ptr(u), _ptr(y_out), int(precision),
                                  _stream(stream)))
        return y_out


class Batch:
    """Many IBDL solves in one persistent launch (``ibdl_solve_batched``)."""

    def __init__(self, capacity):
        h = C.c_void_p()
        _check(load().ibdl_batch_create(int(capacity), C.byref(h)))
        self._h = h
        self.capacity = int(capacity)

    def close(self):
        if getattr(self, "_h", None):
            load().ibdl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, geoms, bdata, q_out, tol=1e-8, restart=30, max_iters=500, max_refine=8,
              inner_tol=1e-5, stream=None, raise_on_error=True):
        n = len(geoms)
        o = SolveOpts()
        load().ibdl_solve_opts_default(C.byref(o))
        o.tol, o.restart, o.max_iters = float(tol), int(restart), int(max_iters)
        o.max_refine, o.inner_tol = int(max_refine), float(inner_tol)
        G = (C.c_void_p * n)(*[g._h.value for g in geoms])
        B = (C.c_void_p * n)(*[_ptr(b) for b in bdata])
        Q = (C.c_void_p * n)(*[_ptr(q) for q in q_out])
        infos = (SolveInfo * n)()
        sts = (C.c_int * n)()
        st = load().ibdl_solve_batched(self._h, n, G, B, Q, C.byref(o), infos, sts,
                                       _stream(stream))
        if raise_on_error:
            _check(st)
        out = []
        for k in range(n):
            d = infos[k].as_dict()
            d["status"] = int(sts[k])
            out.append(d)
        return out
