"""Python binding of libstokes_gb300 (the C ABI of include/stokes.h).

Argument marshalling only: every function forwards device pointers of torch
CUDA tensors (float64, contiguous) and the current torch CUDA stream to the
library of the same name.  There is no CPU fallback: importing this module
raises if the shared library has not been built, and every call raises
``StokesError`` on a non-zero return code (except ``stk_solve`` returning
``STK_ERR_NOT_CONVERGED``, which is reported through the info record).

Layouts: a cell array has shape (nz, ny, nx) (nz = 1 in 2D); the face array
of velocity component a has the same shape with n_a + 1 entries along axis a
when that axis has walls (wall faces hold zeros).  ``face_shape`` gives them.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# STK_LIBRARY selects another build of the library (e.g. the bounds-checked
# libstokes_gb300_check.so); the default is the release build beside this file
LIB_PATH = os.environ.get("STK_LIBRARY") or os.path.join(HERE, "libstokes_gb300.so")

STK_PERIODIC, STK_NOSLIP, STK_FREESLIP = 0, 1, 2
STK_OK = 0
STK_ERR_ARG, STK_ERR_SIZE, STK_ERR_CUDA, STK_ERR_NOT_CONVERGED = -1, -2, -3, -4
STK_ERR_NONFINITE, STK_ERR_TIMEOUT, STK_ERR_STATE = -5, -6, -7
STK_P1, STK_P2, STK_P3, STK_P4, STK_P5 = 1, 2, 3, 4, 5
STK_FP64, STK_MIXED = 0, 1
STK_NPROF = 24


class StokesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stokes error {code}: {msg}")
        self.code = code


class stk_solver_params(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int), ("restart", ctypes.c_int), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("precision", ctypes.c_int), ("nu", ctypes.c_int),
                ("ncoarse", ctypes.c_int), ("vcycles_u", ctypes.c_int), ("vcycles_p", ctypes.c_int)]


class stk_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("est_residual", ctypes.c_double),
                ("scalar_vcycles", ctypes.c_double), ("solve_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stk_schedule(ctypes.Structure):
    _fields_ = [("coarse_level", ctypes.c_int), ("threads", ctypes.c_int),
                ("pair_level", ctypes.c_int), ("grid_level", ctypes.c_int),
                ("cluster_level", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stk_batch_io(ctypes.Structure):
    _fields_ = [("b_u", ctypes.POINTER(ctypes.c_void_p)), ("b_p", ctypes.c_void_p),
                ("x_u", ctypes.POINTER(ctypes.c_void_p)), ("x_p", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1308_4605_gb300.build`"
                          " (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "stk_default_params": (None, [ctypes.POINTER(stk_solver_params)]),
        "stk_create": (I, [I, ctypes.POINTER(I), D, ctypes.POINTER(I), ctypes.POINTER(P)]),
        "stk_create_stacked": (I, [I, ctypes.POINTER(I), D, ctypes.POINTER(I), I, ctypes.POINTER(P)]),
        "stk_stack_count": (I, [P]),
        "stk_stack_info": (I, [P, I, ctypes.POINTER(stk_solve_info)]),
        "stk_stack_history": (I, [P, I, I, ctypes.POINTER(D), I]),
        "stk_destroy": (I, [P]),
        "stk_last_error": (ctypes.c_char_p, [P]),
        "stk_face_length": (ctypes.c_longlong, [P, I]),
        "stk_cell_length": (ctypes.c_longlong, [P]),
        "stk_set_coefficients": (I, [P, P, P, D, P]),
        "stk_set_bulk_viscosity": (I, [P, P, P]),
        "stk_apply_operator": (I, [P, PP, P, PP, P, P]),
        "stk_apply_preconditioner": (I, [P, I, PP, P, PP, P, P]),
        "stk_apply_preconditioner_params": (I, [P, ctypes.POINTER(stk_solver_params), PP, P, PP, P, P]),
        "stk_velocity_vcycle": (I, [P, PP, PP, P]),
        "stk_pressure_vcycle": (I, [P, P, P, P]),
        "stk_solve": (I, [P, ctypes.POINTER(stk_solver_params), PP, P, PP, P,
                          ctypes.POINTER(stk_solve_info), P]),
        "stk_profile": (I, [P, I]),
        "stk_kernel_launches": (ctypes.c_longlong, [P]),
        "stk_gradient": (I, [P, PP, PP, P, P, P]),
        "stk_backward_euler_rhs": (I, [P, PP, PP, PP, P]),
        "stk_subtract_boundary_terms": (I, [P, PP, ctypes.POINTER(ctypes.c_void_p), PP, P, P]),
        "stk_get_schedule": (I, [P, I, ctypes.POINTER(stk_schedule)]),
        "stk_set_schedule": (I, [P, I, ctypes.POINTER(stk_schedule)]),
        "stk_autotune": (I, [P, I, ctypes.POINTER(stk_schedule), P]),
        "stk_solve_batched": (I, [I, ctypes.POINTER(P), ctypes.POINTER(stk_solver_params),
                                  ctypes.POINTER(stk_batch_io), ctypes.POINTER(stk_solve_info), P]),
        "stk_remove_mean": (I, [P, P, P, P]),
        "stk_set_graphs": (I, [P, I]),
        "stk_graphs_in_use": (I, [P]),
        "stk_widen": (I, [P, P, ctypes.c_longlong, P]),
        "stk_set_wait_budget": (I, [P, ctypes.c_longlong]),
        "stk_wait_status": (I, [P, I]),
        "stk_bounds_violations": (ctypes.c_longlong, [ctypes.POINTER(ctypes.c_longlong),
                                                      ctypes.POINTER(ctypes.c_longlong), I]),
        "stk_bounds_selftest": (I, [P]),
        "stk_solve_history": (I, [P, I, ctypes.POINTER(D), I]),
        "stk_pressure_vcycle_noalloc": (I, [I, ctypes.POINTER(I), D, ctypes.POINTER(I), P, P, P, P]),
        "stk_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ["stk_default_params", "stk_create", "stk_create_stacked", "stk_stack_count", "stk_stack_info",
            "stk_stack_history", "stk_destroy", "stk_last_error", "stk_face_length",
            "stk_cell_length", "stk_set_coefficients", "stk_set_bulk_viscosity", "stk_apply_operator",
            "stk_apply_preconditioner", "stk_apply_preconditioner_params", "stk_velocity_vcycle", "stk_pressure_vcycle", "stk_solve",
            "stk_profile", "stk_profile_read", "stk_kernel_launches", "stk_pressure_vcycle_noalloc", "stk_remove_mean", "stk_set_graphs", "stk_graphs_in_use", "stk_widen", "stk_set_wait_budget", "stk_wait_status", "stk_solve_history", "stk_bounds_violations", "stk_bounds_selftest", "stk_gradient", "stk_backward_euler_rhs", "stk_subtract_boundary_terms", "stk_solve_batched", "stk_get_schedule", "stk_set_schedule", "stk_autotune"]


def library():
    return _lib


def _check(h, rc):
    if rc != STK_OK:
        msg = _lib.stk_last_error(h)
        raise StokesError(rc, msg.decode() if msg else "")
    return rc


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, numel=None, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if t.dtype != (dtype or torch.float64):
        raise TypeError(f"expected {dtype or torch.float64}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _ptrs(ts, lengths):
    arr = (ctypes.c_void_p * 3)()
    for a, (t, n) in enumerate(zip(ts, lengths)):
        arr[a] = _ptr(t, n).value
    return arr


def face_shape(n, bc, a):
    ext = list(n) + [1] * (3 - len(n))
    if bc[2 * a] != STK_PERIODIC:
        ext[a] += 1
    return (ext[2], ext[1], ext[0])


# ------------------------------------------------------------- C ABI mirrors
def stk_default_params():
    p = stk_solver_params()
    _lib.stk_default_params(ctypes.byref(p))
    return p


def stk_create(dim, n, h, bc):
    nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    bb = (ctypes.c_int * 6)(*(list(bc) + [0] * (6 - len(bc))))
    out = ctypes.c_void_p()
    _check(None, _lib.stk_create(int(dim), nn, float(h), bb, ctypes.byref(out)))
    return out


def stk_create_stacked(dim, n, h, bc, count):
    nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    bb = (ctypes.c_int * 6)(*(list(bc) + [0] * (6 - len(bc))))
    out = ctypes.c_void_p()
    _check(None, _lib.stk_create_stacked(int(dim), nn, float(h), bb, int(count), ctypes.byref(out)))
    return out


def stk_stack_count(h):
    return int(_lib.stk_stack_count(h))


def stk_stack_info(h, instance):
    info = stk_solve_info()
    _check(h, _lib.stk_stack_info(h, int(instance), ctypes.byref(info)))
    return info.as_dict()


def stk_stack_history(h, instance, kind):
    n = int(_lib.stk_stack_history(h, int(instance), int(kind), None, 0))
    if n < 0:
        raise StokesError(n, "stk_stack_history failed")
    buf = (ctypes.c_double * max(n, 1))()
    got = int(_lib.stk_stack_history(h, int(instance), int(kind), buf, n))
    return [buf[i] for i in range(min(n, got))]


def stk_destroy(h):
    return _check(h, _lib.stk_destroy(h))


def stk_last_error(h):
    m = _lib.stk_last_error(h)
    return m.decode() if m else ""


def stk_face_length(h, a):
    return int(_lib.stk_face_length(h, a))


def stk_cell_length(h):
    return int(_lib.stk_cell_length(h))


def _lengths(h, dim):
    return [stk_face_length(h, a) for a in range(dim)], stk_cell_length(h)


def stk_set_coefficients(h, rho, mu, dt, stream=None):
    nc = stk_cell_length(h)
    return _check(h, _lib.stk_set_coefficients(h, _ptr(rho, nc), _ptr(mu, nc), float(dt),
                                               _stream(stream)))


def stk_set_bulk_viscosity(h, gamma, stream=None):
    nc = int(_lib.stk_cell_length(h))
    return _check(h, _lib.stk_set_bulk_viscosity(h, _ptr(gamma, nc) if gamma is not None else None,
                                                 _stream(stream)))


def stk_apply_operator(h, x_u, x_p, y_u, y_p, stream=None):
    fl, nc = _lengths(h, len(x_u))
    return _check(h, _lib.stk_apply_operator(h, _ptrs(x_u, fl), _ptr(x_p, nc), _ptrs(y_u, fl),
                                             _ptr(y_p, nc), _stream(stream)))


def stk_apply_preconditioner(h, which, b_u, b_p, x_u, x_p, stream=None):
    fl, nc = _lengths(h, len(b_u))
    return _check(h, _lib.stk_apply_preconditioner(h, int(which), _ptrs(b_u, fl), _ptr(b_p, nc),
                                                   _ptrs(x_u, fl), _ptr(x_p, nc), _stream(stream)))


def stk_apply_preconditioner_params(h, params, b_u, b_p, x_u, x_p, stream=None):
    fl, nc = _lengths(h, len(b_u))
    return _check(h, _lib.stk_apply_preconditioner_params(
        h, ctypes.byref(params), _ptrs(b_u, fl), _ptr(b_p, nc), _ptrs(x_u, fl), _ptr(x_p, nc),
        _stream(stream)))


def stk_subtract_boundary_terms(h, u_wall, u_tan, b_u, b_p, stream=None):
    """b -= boundary terms.  u_wall: list of face arrays (wall entries used)
    or None; u_tan: dict {(d, side, a): array} of tangential wall velocities
    or None (see stokes.h)."""
    fl, nc = _lengths(h, len(b_u))
    uw = _ptrs(u_wall, fl) if u_wall is not None else None
    ut = None
    keep = []
    if u_tan:
        ut = (ctypes.c_void_p * 18)()
        for (d, side, a), t in u_tan.items():
            keep.append(t)
            ut[3 * (2 * d + side) + a] = _ptr(t).value
    return _check(h, _lib.stk_subtract_boundary_terms(h, uw, ut, _ptrs(b_u, fl), _ptr(b_p, nc),
                                                      _stream(stream)))


def stk_backward_euler_rhs(h, u_n, f, b_u, stream=None):
    fl, _ = _lengths(h, len(u_n))
    fp = _ptrs(f, fl) if f is not None else None
    return _check(h, _lib.stk_backward_euler_rhs(h, _ptrs(u_n, fl), fp, _ptrs(b_u, fl),
                                                 _stream(stream)))


def stk_velocity_vcycle(h, r_u, x_u, stream=None):
    fl, _ = _lengths(h, len(r_u))
    return _check(h, _lib.stk_velocity_vcycle(h, _ptrs(r_u, fl), _ptrs(x_u, fl), _stream(stream)))


def stk_pressure_vcycle(h, r_p, x_p, stream=None):
    nc = stk_cell_length(h)
    return _check(h, _lib.stk_pressure_vcycle(h, _ptr(r_p, nc), _ptr(x_p, nc), _stream(stream)))


def stk_solve(h, params, b_u, b_p, x_u, x_p, stream=None):
    """Returns the info record as a dict; raises unless converged or
    STK_ERR_NOT_CONVERGED."""
    fl, nc = _lengths(h, len(b_u))
    info = stk_solve_info()
    rc = _lib.stk_solve(h, ctypes.byref(params), _ptrs(b_u, fl), _ptr(b_p, nc), _ptrs(x_u, fl),
                        _ptr(x_p, nc), ctypes.byref(info), _stream(stream))
    if rc not in (STK_OK, STK_ERR_NOT_CONVERGED):
        _check(h, rc)
    return info.as_dict()


def stk_solve_batched(handles, params, b_us, b_ps, x_us, x_ps, stream=None):
    """Solve len(handles) independent systems together (see stokes.h).
    Returns the list of info dicts; raises unless every solve converged or
    the only failure is STK_ERR_NOT_CONVERGED."""
    count = len(handles)
    hs = (ctypes.c_void_p * count)(*[h.value for h in handles])
    keep = []
    ios = (stk_batch_io * count)()
    for i, h in enumerate(handles):
        dim = len(b_us[i])
        fl, nc = _lengths(h, dim)
        bu, xu = _ptrs(b_us[i], fl), _ptrs(x_us[i], fl)
        keep += [bu, xu]
        ios[i].b_u = ctypes.cast(bu, ctypes.POINTER(ctypes.c_void_p))
        ios[i].b_p = _ptr(b_ps[i], nc)
        ios[i].x_u = ctypes.cast(xu, ctypes.POINTER(ctypes.c_void_p))
        ios[i].x_p = _ptr(x_ps[i], nc)
    infos = (stk_solve_info * count)()
    rc = _lib.stk_solve_batched(count, hs, ctypes.byref(params), ios, infos, _stream(stream))
    if rc not in (STK_OK, STK_ERR_NOT_CONVERGED):
        bad = [i for i in range(count) if infos[i].status not in (STK_OK, STK_ERR_NOT_CONVERGED)]
        _check(handles[bad[0]] if bad else None, rc)
    return [infos[i].as_dict() for i in range(count)]


def stk_get_schedule(h, precision):
    sc = stk_schedule()
    _check(h, _lib.stk_get_schedule(h, int(precision), ctypes.byref(sc)))
    return sc.as_dict()


def stk_set_schedule(h, precision, coarse_level, threads, pair_level, grid_level=None,
                     cluster_level=None):
    """grid_level / cluster_level None: no persistent multi-block / cluster
    levels (= coarse_level)."""
    gl = coarse_level if grid_level is None else grid_level
    cl = coarse_level if cluster_level is None else cluster_level
    sc = stk_schedule(int(coarse_level), int(threads), int(pair_level), int(gl), int(cl))
    return _check(h, _lib.stk_set_schedule(h, int(precision), ctypes.byref(sc)))


def stk_autotune(h, precision, stream=None):
    sc = stk_schedule()
    _check(h, _lib.stk_autotune(h, int(precision), ctypes.byref(sc), _stream(stream)))
    return sc.as_dict()


def stk_profile(h, enable):
    return _check(h, _lib.stk_profile(h, int(enable)))


def stk_pressure_vcycle_noalloc(dim, n, h, bc, rho, r_p, x_p, stream=None):
    """One pressure V-cycle without any device allocation (see stokes.h)."""
    nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    bb = (ctypes.c_int * 6)(*(list(bc) + [0] * (6 - len(bc))))
    ncell = int(nn[0]) * int(nn[1]) * int(nn[2])
    rc = _lib.stk_pressure_vcycle_noalloc(int(dim), nn, float(h), bb, _ptr(rho, ncell),
                                          _ptr(r_p, ncell), _ptr(x_p, ncell), _stream(stream))
    if rc != STK_OK:
        raise StokesError(rc, "stk_pressure_vcycle_noalloc failed")
    return rc


def stk_gradient(h, u, lam, dlogmu, drho, stream=None):
    fl, nc = _lengths(h, len(u))
    return _check(h, _lib.stk_gradient(h, _ptrs(u, fl), _ptrs(lam, fl), _ptr(dlogmu, nc), _ptr(drho, nc),
                                       _stream(stream)))


def stk_remove_mean(h, x_p, y_p, stream=None):
    nc = stk_cell_length(h)
    return _check(h, _lib.stk_remove_mean(h, _ptr(x_p, nc), _ptr(y_p, nc), _stream(stream)))


def stk_solve_history(h, kind):
    """Residual history of the last solve on h: kind 0 the true relative
    residual at every cycle start, kind 1 the Arnoldi estimates (stokes.h)."""
    n = int(_lib.stk_solve_history(h, int(kind), None, 0))
    if n < 0:
        raise StokesError(n, "stk_solve_history failed")
    buf = (ctypes.c_double * max(n, 1))()
    got = int(_lib.stk_solve_history(h, int(kind), buf, n))
    return [buf[i] for i in range(min(n, got))]


def stk_bounds_violations(reset=False):
    """(count, first kind, first index) of out-of-range indices met by a
    bounds-checked build; count -1 for a release build."""
    k, i = ctypes.c_longlong(0), ctypes.c_longlong(0)
    n = int(_lib.stk_bounds_violations(ctypes.byref(k), ctypes.byref(i), int(bool(reset))))
    return n, k.value, i.value


def stk_bounds_selftest(stream=None):
    return _check(None, _lib.stk_bounds_selftest(_stream(stream)))


def stk_set_graphs(h, enable):
    return _check(h, _lib.stk_set_graphs(h, int(bool(enable))))


def stk_widen(x, y, stream=None):
    """y (float64) = x (float32), the library's exact widening."""
    import torch
    n = x.numel()
    rc = _lib.stk_widen(_ptr(x, n, dtype=torch.float32), _ptr(y, n), n, _stream(stream))
    if rc != STK_OK:
        raise StokesError(rc, "stk_widen failed")
    return rc


def stk_graphs_in_use(h):
    return int(_lib.stk_graphs_in_use(h))


def stk_set_wait_budget(h, cycles):
    return _check(h, _lib.stk_set_wait_budget(h, int(cycles)))


def stk_wait_status(h, reset=False):
    """STK_OK, or STK_ERR_TIMEOUT when a bounded device wait ran out."""
    return int(_lib.stk_wait_status(h, int(bool(reset))))


def stk_kernel_launches(h):
    return int(_lib.stk_kernel_launches(h))


def stk_profile_read(h, k):
    name = ctypes.c_char_p()
    launches = ctypes.c_longlong()
    ms = ctypes.c_double()
    nbytes = ctypes.c_double()
    flops = ctypes.c_double()
    rc = _lib.stk_profile_read(h, int(k), ctypes.byref(name), ctypes.byref(launches),
                               ctypes.byref(ms), ctypes.byref(nbytes), ctypes.byref(flops))
    if rc != 0:
        raise StokesError(rc, "profile index out of range")
    return {"name": name.value.decode(), "launches": launches.value, "ms": ms.value,
            "bytes": nbytes.value, "flops": flops.value}


# ------------------------------------------------------------ convenience
class StokesSolver:
    """Owns one stk_handle; methods take/return torch CUDA tensors.

    count: a stacked batch of `count` 2D instances of the grid
    (stk_create_stacked); every array then has the instances along its
    leading axis (face_shape / cell_shape give (count, ny, nx)-shaped arrays)."""

    def __init__(self, dim, n, bc, h=1.0, count=None):
        self.dim = int(dim)
        self.count = int(count) if count is not None else 1
        self.n = tuple(list(n[:self.dim]) + [1] * (3 - self.dim))
        if count is not None:
            if self.dim != 2:
                raise ValueError("stacked batches are 2D")
            self.n = (self.n[0], self.n[1], self.count)
        self.bc = tuple(list(bc) + [0] * (6 - len(bc)))
        self.h = float(h)
        if count is not None:
            self.handle = stk_create_stacked(dim, n[:2], h, bc, self.count)
        else:
            self.handle = stk_create(dim, n, h, bc)

    def close(self):
        if self.handle is not None and self.handle.value:
            stk_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def face_shape(self, a):
        return face_shape(self.n, self.bc, a)

    def cell_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def zeros(self, device="cuda"):
        import torch
        u = [torch.zeros(self.face_shape(a), dtype=torch.float64, device=device) for a in range(self.dim)]
        p = torch.zeros(self.cell_shape(), dtype=torch.float64, device=device)
        return u, p

    def set_coefficients(self, rho, mu, theta):
        dt = math.inf if theta == 0.0 else 1.0 / theta
        stk_set_coefficients(self.handle, rho, mu, dt)

    def subtract_boundary_terms(self, b_u, b_p, u_wall=None, u_tan=None):
        """b -= the boundary terms of inhomogeneous velocity boundary
        conditions (stk_subtract_boundary_terms); u_tan arrays are checked
        against the a-face extents without axis d."""
        if u_tan:
            for (d, side, a), t in u_tan.items():
                ext = list(face_shape(self.n, self.bc, a))[::-1]   # (x, y, z)
                want = 1
                for c in range(3):
                    if c != d:
                        want *= ext[c]
                if d == a or not (0 <= d < self.dim) or self.bc[2 * d + side] == STK_PERIODIC:
                    raise ValueError(f"no tangential data for wall {(d, side)} and component {a}")
                if t.numel() != want:
                    raise ValueError(f"tangential data {(d, side, a)}: {t.numel()} values, expected {want}")
        stk_subtract_boundary_terms(self.handle, u_wall, u_tan, b_u, b_p)

    def set_bulk_viscosity(self, gamma):
        """gamma: cell array of bulk viscosities, or None to switch off."""
        stk_set_bulk_viscosity(self.handle, gamma)

    def apply_operator(self, x_u, x_p):
        y_u, y_p = self.zeros(x_p.device)
        stk_apply_operator(self.handle, x_u, x_p, y_u, y_p)
        return y_u, y_p

    def apply_preconditioner(self, which, b_u, b_p, **kw):
        """x = P_which^{-1} b; keyword arguments (precision, nu, ncoarse,
        vcycles_u, vcycles_p) select stk_apply_preconditioner_params."""
        x_u, x_p = self.zeros(b_p.device)
        if kw:
            p = stk_default_params()
            p.precond = int(which)
            for k, v in kw.items():
                setattr(p, k, v)
            stk_apply_preconditioner_params(self.handle, p, b_u, b_p, x_u, x_p)
        else:
            stk_apply_preconditioner(self.handle, which, b_u, b_p, x_u, x_p)
        return x_u, x_p

    def solve(self, b_u, b_p, x_u=None, x_p=None, **kw):
        p = stk_default_params()
        for k, v in kw.items():
            setattr(p, k, v)
        if x_u is None:
            x_u, x_p = self.zeros(b_p.device)
        info = stk_solve(self.handle, p, b_u, b_p, x_u, x_p)
        return x_u, x_p, info

    def instance_info(self, i):
        """The last solve's record of instance i of a stacked batch."""
        return stk_stack_info(self.handle, i)
