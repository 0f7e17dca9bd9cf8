"""Thin ctypes binding of libsdg (include/sdg.h): same names, argument
marshalling only.  Every computation runs in the CUDA library.

Tensors passed to the binding are torch CUDA tensors (device memory and the
current stream come from PyTorch); host arrays for sdg_set_state /
sdg_get_state may also be numpy arrays or CPU tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdg.so")

SDG_OK = 0
SDG_ERR_INVALID_ARG = 1
SDG_ERR_CUDA = 2
SDG_ERR_NOT_CONVERGED = 3
SDG_ERR_BREAKDOWN = 4
SDG_ERR_UNSUPPORTED = 5
SDG_FP64 = 0
SDG_MIXED = 1

# every symbol include/sdg.h declares
EXPORTS = (
    "sdg_nodes", "sdg_matrices", "sdg_kernel_projector", "sdg_line_operator", "sdg_create", "sdg_destroy", "sdg_set_options",
    "sdg_set_mixed_options", "sdg_set_convection_substeps", "sdg_set_iteration_form", "sdg_set_tile", "sdg_autotune", "sdg_ndof", "sdg_set_state", "sdg_get_state",
    "sdg_pressure_apply", "sdg_viscous_apply", "sdg_pressure_cg", "sdg_viscous_cg",
    "sdg_dual_to_main", "sdg_main_to_dual", "sdg_convect", "sdg_pressure_rhs",
    "sdg_velocity_update", "sdg_step", "sdg_step_adjoint", "sdg_set_profiling", "sdg_counters", "sdg_diagnostics",
    "sdg_kinetic_energy_noalloc", "sdg_batch_create", "sdg_batch_destroy", "sdg_batch_size",
    "sdg_batch_member", "sdg_batch_set_threads", "sdg_batch_step", "sdg_strerror", "sdg_last_error",
)


class sdg_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3)]


class sdg_cg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("applies_fp64", ctypes.c_int), ("applies_fp32", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("status", ctypes.c_int), ("true_res", ctypes.c_double),
                ("floor_res", ctypes.c_double), ("eval_res", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sdg_step_info(ctypes.Structure):
    _fields_ = [("pressure", sdg_cg_info), ("viscous", sdg_cg_info * 3),
                ("pressure_ms", ctypes.c_double), ("step_ms", ctypes.c_double),
                ("pressure_applies", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong)]


class SDGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sdg status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libsdg.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1602_05806_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.sdg_nodes.argtypes = [ip, dp, dp]
        L.sdg_matrices.argtypes = [ip, dp]
        L.sdg_kernel_projector.argtypes = [ip, dp, ctypes.POINTER(ctypes.c_int)]
        L.sdg_line_operator.argtypes = [ip, ip, dp, dp, dp]
        L.sdg_create.argtypes = [ctypes.POINTER(sdg_grid), ip, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.POINTER(vp)]
        L.sdg_destroy.argtypes = [vp]
        L.sdg_set_options.argtypes = [vp, ip, ctypes.c_double, ctypes.c_double, ip]
        L.sdg_set_mixed_options.argtypes = [vp, ctypes.c_double, ip, ip]
        L.sdg_set_convection_substeps.argtypes = [vp, ip]
        L.sdg_set_tile.argtypes = [vp, ip]
        L.sdg_set_iteration_form.argtypes = [vp, ip]
        L.sdg_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp, vp]
        L.sdg_ndof.argtypes = [vp]
        L.sdg_ndof.restype = ctypes.c_longlong
        L.sdg_set_state.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sdg_get_state.argtypes = [vp, vp, vp, vp, vp, vp]
        for f in ("sdg_pressure_apply", "sdg_viscous_apply"):
            getattr(L, f).argtypes = [vp, vp, vp, ip, vp]
        for f in ("sdg_pressure_cg", "sdg_viscous_cg"):
            getattr(L, f).argtypes = [vp, vp, vp, ctypes.POINTER(sdg_cg_info), vp]
        for f in ("sdg_dual_to_main", "sdg_main_to_dual"):
            getattr(L, f).argtypes = [vp, ip, vp, vp, vp]
        L.sdg_convect.argtypes = [vp, vp, vp, vp]
        L.sdg_pressure_rhs.argtypes = [vp, vp, vp, vp, vp]
        L.sdg_velocity_update.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sdg_step.argtypes = [vp, ip, ctypes.POINTER(sdg_step_info), vp]
        L.sdg_diagnostics.argtypes = [vp, dp, dp, vp]
        L.sdg_set_profiling.argtypes = [vp, ip]
        L.sdg_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), dp,
                                   ctypes.POINTER(ctypes.c_longlong)]
        L.sdg_kinetic_energy_noalloc.argtypes = [ctypes.POINTER(sdg_grid), ip, vp, vp, vp, vp, vp]
        L.sdg_strerror.argtypes = [ip]
        L.sdg_strerror.restype = ctypes.c_char_p
        L.sdg_last_error.restype = ctypes.c_char_p
        L.sdg_step_adjoint.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
        L.sdg_batch_create.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp, ip, ctypes.c_double,
                                       ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]
        L.sdg_batch_destroy.argtypes = [vp]
        L.sdg_batch_size.argtypes = [vp]
        L.sdg_batch_member.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_void_p)]
        L.sdg_batch_set_threads.argtypes = [vp, ip]
        L.sdg_batch_step.argtypes = [vp, ip, vp, vp]
        for f in EXPORTS:
            if f not in ("sdg_ndof", "sdg_strerror", "sdg_last_error"):
                getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def check(rc, ok=(SDG_OK,)):
    if rc not in ok:
        L = lib()
        detail = L.sdg_last_error().decode() or L.sdg_strerror(rc).decode()
        raise SDGError(rc, detail)
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    """CUDA stream handle: the current torch stream (None), a torch.cuda.Stream,
    or a raw handle."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _ptr_array(ts):
    arr = (ctypes.c_void_p * 3)()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t)
    return arr


# ----------------------------------------------------------------- free functions
def sdg_nodes(N):
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    check(lib().sdg_nodes(N, xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return xi, w


def sdg_matrices(N):
    """dict of the 1D matrices of degree N as computed by the library."""
    m = (N + 1) ** 2
    out = np.zeros(10 * m)
    check(lib().sdg_matrices(N, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    names = ("M", "Rt", "Lt", "Rb", "Lb", "ML", "MR", "HR", "HL", "HC")
    return {k: out[i * m:(i + 1) * m].reshape(N + 1, N + 1).copy() for i, k in enumerate(names)}


def sdg_line_operator(N, fp32=False):
    """(HL, Mc, HR): the stored 1D line operator of the accurate contraction
    in FP64 or FP32, evaluated on the host (see include/sdg.h)."""
    n1 = N + 1
    out = [np.zeros((n1, n1)) for _ in range(3)]
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(lib().sdg_line_operator(N, 1 if fp32 else 0, ptr(out[0]), ptr(out[1]), ptr(out[2])))
    return tuple(out)


def sdg_kernel_projector(N):
    """(projector onto ker(R~ - L~) as an (N+1)x(N+1) array, its dimension)."""
    P = np.zeros((N + 1) * (N + 1))
    d = ctypes.c_int()
    check(lib().sdg_kernel_projector(N, P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(d)))
    return P.reshape(N + 1, N + 1), d.value


def sdg_kinetic_energy_noalloc(dim, n, L, N, U, ke, stream=None):
    """Kinetic energy of device velocity arrays U (dim tensors) into the
    one-element device tensor `ke`, without any device allocation."""
    g = sdg_grid()
    g.dim = dim
    for d in range(3):
        g.n[d] = int(n[d]) if d < dim else 1
        g.L[d] = float(L[d]) if d < dim else 1.0
    w = U[2] if dim == 3 else None
    check(lib().sdg_kinetic_energy_noalloc(ctypes.byref(g), int(N), _ptr(U[0]), _ptr(U[1]), _ptr(w),
                                           _ptr(ke), _stream(stream)))


class Handle:
    """Owns one sdg_handle.  Method names follow the C ABI without the prefix."""

    def __init__(self, dim, n, L, N, nu, theta, dt):
        g = sdg_grid()
        g.dim = dim
        for d in range(3):
            g.n[d] = int(n[d]) if d < dim else 1
            g.L[d] = float(L[d]) if d < dim else 1.0
        h = ctypes.c_void_p()
        check(lib().sdg_create(ctypes.byref(g), int(N), float(nu), float(theta), float(dt), ctypes.byref(h)))
        self.h = h
        self.dim, self.n, self.L, self.N = dim, tuple(n[:dim]), tuple(L[:dim]), N
        self.nu, self.theta, self.dt = nu, theta, dt
        self.ndof = int(lib().sdg_ndof(h))

    _owned = True

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                lib().sdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return tuple(reversed(self.n)) + (self.N + 1,) * self.dim

    def set_options(self, precision=SDG_FP64, rtol_p=1e-12, rtol_v=1e-12, maxit=1000000):
        check(lib().sdg_set_options(self.h, precision, rtol_p, rtol_v, maxit))

    def set_mixed_options(self, delta=0.5, max_updates=10000, deflate=False):
        check(lib().sdg_set_mixed_options(self.h, delta, max_updates, 1 if deflate else 0))

    def set_convection_substeps(self, nsub):
        """SSP-RK3 sub-steps of the explicit convection per time step."""
        check(lib().sdg_set_convection_substeps(self.h, int(nsub)))

    def set_iteration_form(self, form):
        """0: one launch per CG iteration; 1: operator + update launches, x += alpha p in the update;
        2 (default): operator + update launches, x += alpha p in the next operator launch."""
        check(lib().sdg_set_iteration_form(self.h, int(form)))

    def set_tile(self, variant):
        """Tile shape of the 2D FP32 operator (0 base, 1 wide in x, 2 wide in y)."""
        check(lib().sdg_set_tile(self.h, int(variant)))

    def autotune(self, stream=None):
        """(chosen tile variant, mean launch time in us of every variant)."""
        v = ctypes.c_int()
        us = (ctypes.c_double * 3)()
        check(lib().sdg_autotune(self.h, ctypes.byref(v), us, _stream(stream)))
        return v.value, [us[i] for i in range(3 if self.dim == 2 else 2)]

    def set_profiling(self, enable=True):
        check(lib().sdg_set_profiling(self.h, 1 if enable else 0))

    def counters(self):
        n = ctypes.c_longlong()
        ms = (ctypes.c_double * 2)()
        cnt = (ctypes.c_longlong * 2)()
        check(lib().sdg_counters(self.h, ctypes.byref(n), ms, cnt))
        return {"launches": n.value, "apply_ms": [ms[0], ms[1]], "apply_launches": [cnt[0], cnt[1]]}

    def set_state(self, U, P, stream=None):
        w = U[2] if self.dim == 3 else None
        check(lib().sdg_set_state(self.h, _ptr(U[0]), _ptr(U[1]), _ptr(w), _ptr(P), _stream(stream)))

    def get_state(self, U, P, stream=None):
        w = U[2] if self.dim == 3 else None
        check(lib().sdg_get_state(self.h, _ptr(U[0]), _ptr(U[1]), _ptr(w), _ptr(P), _stream(stream)))

    def pressure_apply(self, x, y, stream=None):
        import torch
        fp32 = 1 if x.dtype == torch.float32 else 0
        check(lib().sdg_pressure_apply(self.h, _ptr(x), _ptr(y), fp32, _stream(stream)))

    def viscous_apply(self, x, y, stream=None):
        import torch
        fp32 = 1 if x.dtype == torch.float32 else 0
        check(lib().sdg_viscous_apply(self.h, _ptr(x), _ptr(y), fp32, _stream(stream)))

    def pressure_cg(self, b, x, stream=None, ok=(SDG_OK,)):
        info = sdg_cg_info()
        check(lib().sdg_pressure_cg(self.h, _ptr(b), _ptr(x), ctypes.byref(info), _stream(stream)), ok)
        return info.as_dict()

    def viscous_cg(self, b, x, stream=None, ok=(SDG_OK,)):
        info = sdg_cg_info()
        check(lib().sdg_viscous_cg(self.h, _ptr(b), _ptr(x), ctypes.byref(info), _stream(stream)), ok)
        return info.as_dict()

    def dual_to_main(self, d, x, y, stream=None):
        check(lib().sdg_dual_to_main(self.h, d, _ptr(x), _ptr(y), _stream(stream)))

    def main_to_dual(self, d, x, y, stream=None):
        check(lib().sdg_main_to_dual(self.h, d, _ptr(x), _ptr(y), _stream(stream)))

    def convect(self, V, F, stream=None):
        check(lib().sdg_convect(self.h, _ptr_array(V), _ptr_array(F), _stream(stream)))

    def pressure_rhs(self, Ustar, P_old, b, stream=None):
        check(lib().sdg_pressure_rhs(self.h, _ptr_array(Ustar), _ptr(P_old), _ptr(b), _stream(stream)))

    def velocity_update(self, Ustar, P_new, P_old, U, stream=None):
        check(lib().sdg_velocity_update(self.h, _ptr_array(Ustar), _ptr(P_new), _ptr(P_old),
                                        _ptr_array(U), _stream(stream)))

    def step(self, nsteps=1, stream=None, ok=(SDG_OK,)):
        info = sdg_step_info()
        rc = check(lib().sdg_step(self.h, nsteps, ctypes.byref(info), _stream(stream)), ok)
        return {"status": rc, "pressure": info.pressure.as_dict(),
                "viscous": [info.viscous[c].as_dict() for c in range(self.dim)],
                "pressure_ms": info.pressure_ms, "step_ms": info.step_ms,
                "pressure_applies": info.pressure_applies, "kernel_launches": info.kernel_launches}

    def step_adjoint(self, U, lamU, lamP, stream=None, ok=(SDG_OK,)):
        """Adjoint of one step at the checkpoint U (start of the step):
        lamU / lamP are updated in place from the cotangents of the step's
        outputs to those of its inputs; returns d loss / d nu of the step."""
        dnu = ctypes.c_double(0.0)
        check(lib().sdg_step_adjoint(self.h, _ptr_array(U), _ptr_array(lamU), _ptr(lamP), ctypes.byref(dnu),
                                     _stream(stream)), ok)
        return dnu.value

    def diagnostics(self, stream=None):
        ke = ctypes.c_double()
        dv = ctypes.c_double()
        check(lib().sdg_diagnostics(self.h, ctypes.byref(ke), ctypes.byref(dv), _stream(stream)))
        return ke.value, dv.value


def _step_info_dict(info, dim, rc):
    return {"status": rc, "pressure": info.pressure.as_dict(),
            "viscous": [info.viscous[c].as_dict() for c in range(dim)],
            "pressure_ms": info.pressure_ms, "step_ms": info.step_ms,
            "pressure_applies": info.pressure_applies, "kernel_launches": info.kernel_launches}


class Batch:
    """Owns an sdg_batch of independent 2D/3D problems.  members[i] is a
    non-owning Handle view of member i."""

    def __init__(self, problems, theta, dt):
        """problems: list of (dim, n, L, N, nu)."""
        k = len(problems)
        grids = (sdg_grid * k)()
        Ns = (ctypes.c_int * k)()
        nus = (ctypes.c_double * k)()
        for i, (dim, n, L, N, nu) in enumerate(problems):
            grids[i].dim = dim
            for d in range(3):
                grids[i].n[d] = int(n[d]) if d < dim else 1
                grids[i].L[d] = float(L[d]) if d < dim else 1.0
            Ns[i] = int(N)
            nus[i] = float(nu)
        b = ctypes.c_void_p()
        check(lib().sdg_batch_create(grids, Ns, nus, k, float(theta), float(dt), ctypes.byref(b)))
        self.b = b
        self.members = []
        for i, (dim, n, L, N, nu) in enumerate(problems):
            h = ctypes.c_void_p()
            check(lib().sdg_batch_member(b, i, ctypes.byref(h)))
            m = Handle.__new__(Handle)
            m.h, m._owned = h, False
            m.dim, m.n, m.L, m.N = dim, tuple(n[:dim]), tuple(L[:dim]), N
            m.nu, m.theta, m.dt = nu, theta, dt
            m.ndof = int(lib().sdg_ndof(h))
            self.members.append(m)

    def __len__(self):
        return len(self.members)

    def set_threads(self, n):
        check(lib().sdg_batch_set_threads(self.b, int(n)))

    def step(self, nsteps=1, stream=None, ok=(SDG_OK,)):
        k = len(self.members)
        info = (sdg_step_info * k)()
        rc = check(lib().sdg_batch_step(self.b, int(nsteps), info, _stream(stream)), ok)
        return rc, [_step_info_dict(info[i], self.members[i].dim, rc) for i in range(k)]

    def close(self):
        if getattr(self, "b", None):
            for m in self.members:
                m.h = None
            lib().sdg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
