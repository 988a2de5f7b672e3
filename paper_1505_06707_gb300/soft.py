"""ctypes binding of ``include/soft.h`` (argument marshalling only).

Device buffers are passed as integers (``tensor.data_ptr()``) or as torch
tensors; streams as ``torch.cuda.Stream`` / raw handles / None.  Every
function raises ``SoftError`` on a non-zero status, except the PCG solve,
which returns its status for NOT_CONVERGED so that callers can inspect the
partial result."""
from __future__ import annotations

import ctypes as C
import os

__all__ = [
    "SoftError", "SOFT_C64", "SOFT_C128", "CONTOUR_SHARP", "CONTOUR_SECS", "CONTOUR_TFECS",
    "ABSORB_CAP", "ABSORB_TFAP",
    "load", "lib_path", "exported_symbols", "Options", "Field", "soft_create", "soft_create_batch",
    "soft_batch_layout", "soft_step", "soft_step_batch", "soft_step_noalloc", "soft_step_status",
    "soft_step_surface", "sse_surff", "soft_observe",
    "soft_set_potential", "sse_pcg_solve",
    "sse_apply_A", "sse_apply_A32", "sse_apply_precond", "soft_destroy", "sse_nn_set_weights", "sse_nn_get_weights",
    "sse_nn_forward", "sse_nn_grad", "sse_nn_train", "NN_PARAMS", "soft_plan_points", "soft_plan_count",
    "soft_last_launches", "Plan",
]

SOFT_C64, SOFT_C128 = 1, 2
CONTOUR_SHARP, CONTOUR_SECS, CONTOUR_TFECS = 0, 1, 2
ABSORB_CAP, ABSORB_TFAP = 3, 4
ERR_NOT_CONVERGED = -5

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libsoft.so")
_lib = None

# every symbol include/soft.h declares
exported_symbols = [
    "soft_default_options", "soft_create", "soft_create_batch", "soft_batch_layout", "soft_step",
    "soft_step_batch", "soft_observe", "soft_set_potential", "sse_pcg_solve", "sse_apply_A", "sse_apply_A32",
    "sse_apply_precond", "soft_destroy", "soft_strerror", "soft_plan_count", "soft_plan_points", "soft_plan_prec",
    "soft_last_launches", "soft_step_noalloc", "soft_step_status", "soft_step_surface", "sse_surff",
    "sse_nn_set_weights", "sse_nn_get_weights",
    "sse_nn_forward", "sse_nn_grad", "sse_nn_train",
]


class SoftError(RuntimeError):
    def __init__(self, status, where):
        msg = load().soft_strerror(status).decode() if _lib is not None else str(status)
        super().__init__("%s failed: %s (%d)" % (where, msg, status))
        self.status = status


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int64 * 3)]


class Options(C.Structure):
    _fields_ = [("prec", C.c_int), ("contour", C.c_int), ("tfecs_alpha", C.c_double),
                ("soft_a2", C.c_double), ("charge", C.c_double), ("band_width", C.c_int),
                ("autotune", C.c_int), ("cap_energy", C.c_double), ("tfap_kmin", C.c_double),
                ("persistent", C.c_int)]


class Field(C.Structure):
    _fields_ = [("E0", C.c_double), ("omega", C.c_double), ("ncycles", C.c_double)]


def lib_path():
    return _LIB_PATH


def load():
    """Load libsoft.so (built by ``__graft_entry__.build()`` or
    ``python -m paper_1505_06707_gb300._build``).  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libsoft.so not built (%s); run the build step first" % _LIB_PATH)
    L = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    i64 = C.c_int64
    dbl = C.c_double
    L.soft_default_options.argtypes = [C.POINTER(Options)]
    L.soft_create.argtypes = [C.POINTER(Grid), C.POINTER(dbl), dbl, dbl, dbl, C.POINTER(Options),
                              C.POINTER(P)]
    L.soft_create_batch.argtypes = [C.c_int, C.POINTER(Grid), C.POINTER(dbl), C.POINTER(dbl),
                                    C.POINTER(dbl), C.POINTER(Field), dbl, C.POINTER(Options),
                                    C.POINTER(P)]
    L.soft_batch_layout.argtypes = [P, C.POINTER(i64), C.POINTER(i64)]
    L.soft_step.argtypes = [P, P, i64, C.POINTER(Field), C.POINTER(dbl), P]
    L.soft_step_batch.argtypes = [P, P, i64, C.POINTER(dbl), P]
    L.soft_step_noalloc.argtypes = [P, P, i64, C.POINTER(Field), C.POINTER(dbl), P]
    L.soft_step_status.argtypes = [P, P]
    L.soft_step_surface.argtypes = [P, P, i64, C.POINTER(Field), C.POINTER(dbl), P, P]
    L.sse_surff.argtypes = [P, C.c_int, C.POINTER(dbl), P, P, i64, dbl, C.c_int, P, P]
    L.soft_observe.argtypes = [P, P, P, P, P]
    L.soft_set_potential.argtypes = [P, P, i64]
    L.sse_pcg_solve.argtypes = [P, C.POINTER(dbl), C.c_int, P, P, dbl, C.c_int, C.c_int,
                                C.POINTER(C.c_int), C.POINTER(dbl), P]
    L.sse_apply_A.argtypes = [P, dbl, P, P, P]
    L.sse_apply_A32.argtypes = [P, dbl, P, P, P]
    L.sse_apply_precond.argtypes = [P, dbl, C.c_int, P, P, P]
    L.sse_nn_set_weights.argtypes = [P, P]
    L.sse_nn_get_weights.argtypes = [P, P]
    L.sse_nn_forward.argtypes = [P, P, C.c_int, C.c_int, C.c_int, P, P]
    L.sse_nn_grad.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, P, C.POINTER(dbl), P]
    L.sse_nn_train.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dbl,
                               C.c_uint64, P, P]
    L.soft_destroy.argtypes = [P]
    L.soft_destroy.restype = None
    L.soft_strerror.argtypes = [C.c_int]
    L.soft_strerror.restype = C.c_char_p
    L.soft_plan_count.argtypes = [P]
    L.soft_plan_points.argtypes = [P, C.c_int]
    L.soft_plan_points.restype = i64
    L.soft_plan_prec.argtypes = [P]
    L.soft_last_launches.argtypes = [P]
    L.soft_last_launches.restype = i64
    for name in exported_symbols:
        if name not in ("soft_destroy", "soft_strerror", "soft_plan_points", "soft_last_launches",
                        "soft_default_options"):
            getattr(L, name).restype = C.c_int
    L.soft_default_options.restype = None
    _lib = L
    return L


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("expected a device pointer or tensor")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, where):
    if rc != 0:
        raise SoftError(rc, where)


def _options(prec=SOFT_C128, contour=CONTOUR_SHARP, tfecs_alpha=0.5, soft_a2=2.0, charge=1.0,
             band_width=10, autotune=0, cap_energy=2.0, tfap_kmin=0.25, persistent=1):
    o = Options()
    load().soft_default_options(C.byref(o))
    o.prec, o.contour, o.tfecs_alpha = prec, contour, tfecs_alpha
    o.soft_a2, o.charge, o.band_width = soft_a2, charge, band_width
    o.autotune = autotune
    o.persistent = persistent
    o.cap_energy, o.tfap_kmin = cap_energy, tfap_kmin
    return o


def soft_create(n, box, R0, theta, dt, **opts):
    """n: int (1D), (nx, ny) or (nx, ny, nz); box: (a, b), (ax, bx, ay, by) or
    (ax, bx, ay, by, az, bz)."""
    L = load()
    g = Grid()
    dims = list(n) if isinstance(n, (tuple, list)) else [n]
    if not 1 <= len(dims) <= 3 or len(box) != 2 * len(dims):
        raise ValueError("soft_create: n and box disagree")
    g.ndim = len(dims)
    for d, v in enumerate(dims):
        g.n[d] = v
    bx = (C.c_double * len(box))(*box)
    o = _options(**opts)
    out = C.c_void_p()
    _check(L.soft_create(C.byref(g), bx, R0, theta, dt, C.byref(o), C.byref(out)), "soft_create")
    return out.value


def soft_create_batch(ns, boxes, R0s, thetas, fields, dt, **opts):
    L = load()
    cnt = len(ns)
    G = (Grid * cnt)()
    for i, n in enumerate(ns):
        G[i].ndim, G[i].n[0] = 1, n
    bx = (C.c_double * (2 * cnt))(*[v for b in boxes for v in b])
    r0 = (C.c_double * cnt)(*R0s)
    th = (C.c_double * cnt)(*thetas)
    F = None
    if fields is not None:
        F = (Field * cnt)()
        for i, f in enumerate(fields):
            if f is not None:
                F[i].E0, F[i].omega, F[i].ncycles = f
    o = _options(**opts)
    out = C.c_void_p()
    _check(L.soft_create_batch(cnt, G, bx, r0, th, F, dt, C.byref(o), C.byref(out)),
           "soft_create_batch")
    return out.value


def soft_batch_layout(plan):
    cnt = load().soft_plan_count(plan)
    off = (C.c_int64 * cnt)()
    tot = C.c_int64()
    _check(load().soft_batch_layout(plan, off, C.byref(tot)), "soft_batch_layout")
    return list(off), tot.value


def soft_step(plan, psi, nsteps, t, field=None, stream=None):
    """Returns the advanced time."""
    tt = C.c_double(t)
    F = None
    if field is not None:
        F = Field(*field)
    _check(load().soft_step(plan, _ptr(psi), int(nsteps), C.byref(F) if F is not None else None,
                            C.byref(tt), _stream(stream)), "soft_step")
    return tt.value


def soft_step_noalloc(plan, psi, nsteps, t, field=None, stream=None):
    """soft_step without any device allocation (fixed scratch, at most 16384
    steps per call).  Returns the advanced time."""
    tt = C.c_double(t)
    F = None
    if field is not None:
        F = Field(*field)
    _check(load().soft_step_noalloc(plan, _ptr(psi), int(nsteps),
                                    C.byref(F) if F is not None else None, C.byref(tt),
                                    _stream(stream)), "soft_step_noalloc")
    return tt.value


def soft_step_batch(plan, psi, nsteps, t, stream=None):
    tt = C.c_double(t)
    _check(load().soft_step_batch(plan, _ptr(psi), int(nsteps), C.byref(tt), _stream(stream)),
           "soft_step_batch")
    return tt.value


def soft_step_status(plan, stream=None):
    """Wait for the stream; raise SoftError(NONFINITE) if a step of this 1D
    plan has produced a non-finite state since the last query."""
    _check(load().soft_step_status(plan, _stream(stream)), "soft_step_status")


def soft_step_surface(plan, psi, nsteps, t, samples, field=None, stream=None):
    """soft_step that also writes psi, dpsi/dx at +R0 and -R0 after every step
    into samples (device complex128 [nsteps + 1][4]).  Returns the time."""
    tt = C.c_double(t)
    F = Field(*field) if field is not None else None
    _check(load().soft_step_surface(plan, _ptr(psi), int(nsteps), C.byref(F) if F is not None else None,
                                    C.byref(tt), _ptr(samples), _stream(stream)), "soft_step_surface")
    return tt.value


def sse_surff(plan, E, phi, samples, t0=0.0, rule=1, amp=None, stream=None):
    """t&E-SURFF amplitudes A(+k), A(-k) for k = sqrt(2E); phi: device
    complex128 [nE][N] from sse_pcg_solve with right-hand side psi(T);
    samples from soft_step_surface.  Returns the device array amp [nE][2]."""
    import torch
    nE = len(E)
    if amp is None:
        amp = torch.zeros((nE, 2), dtype=torch.complex128, device=phi.device)
    Ea = (C.c_double * nE)(*E)
    _check(load().sse_surff(plan, nE, Ea, _ptr(phi), _ptr(samples), int(samples.shape[0]), float(t0),
                            int(rule), _ptr(amp), _stream(stream)), "sse_surff")
    return amp


def soft_observe(plan, psi, norm_in, flux, stream=None):
    _check(load().soft_observe(plan, _ptr(psi), _ptr(norm_in), _ptr(flux), _stream(stream)),
           "soft_observe")


def soft_set_potential(plan, U):
    """U: complex array of the plan's grid shape (host), the potential at
    the complex-scaled grid points."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).ravel())
    _check(load().soft_set_potential(plan, a.ctypes.data, a.size), "soft_set_potential")


def sse_pcg_solve(plan, E, rhs, psi_out, tol=1e-8, maxit=1000, precond=1, stream=None):
    """Returns (status, iterations list, relative residual list)."""
    nE = len(E)
    Ea = (C.c_double * nE)(*E)
    it = (C.c_int * nE)()
    rr = (C.c_double * nE)()
    rc = load().sse_pcg_solve(plan, Ea, nE, _ptr(rhs), _ptr(psi_out), tol, maxit, precond, it, rr,
                              _stream(stream))
    if rc not in (0, ERR_NOT_CONVERGED):
        raise SoftError(rc, "sse_pcg_solve")
    return rc, list(it), list(rr)


def sse_apply_A(plan, E, x, y, stream=None):
    _check(load().sse_apply_A(plan, E, _ptr(x), _ptr(y), _stream(stream)), "sse_apply_A")


def sse_apply_A32(plan, E, x, y, stream=None):
    _check(load().sse_apply_A32(plan, E, _ptr(x), _ptr(y), _stream(stream)), "sse_apply_A32")


def sse_apply_precond(plan, E, precond, x, y, stream=None):
    _check(load().sse_apply_precond(plan, E, precond, _ptr(x), _ptr(y), _stream(stream)),
           "sse_apply_precond")


NN_PARAMS = 10434


def sse_nn_set_weights(plan, w):
    import numpy as np
    a = np.ascontiguousarray(w, dtype=np.float32)
    assert a.size == NN_PARAMS
    _check(load().sse_nn_set_weights(plan, a.ctypes.data), "sse_nn_set_weights")


def sse_nn_get_weights(plan):
    import numpy as np
    a = np.zeros(NN_PARAMS, dtype=np.float32)
    _check(load().sse_nn_get_weights(plan, a.ctypes.data), "sse_nn_get_weights")
    return a


def sse_nn_forward(plan, x, out, stream=None):
    """x: device complex64 [n][H][W]; out: device float32 [n][H][W][2]."""
    n, H, W = x.shape
    _check(load().sse_nn_forward(plan, _ptr(x), n, H, W, _ptr(out), _stream(stream)),
           "sse_nn_forward")


def sse_nn_grad(plan, x, t, stream=None):
    """Returns (loss, gradient float32[10434]) of the mean-square loss."""
    import numpy as np
    n, H, W = x.shape
    g = np.zeros(NN_PARAMS, dtype=np.float32)
    loss = C.c_double()
    _check(load().sse_nn_grad(plan, _ptr(x), _ptr(t), n, H, W, g.ctypes.data, C.byref(loss),
                              _stream(stream)), "sse_nn_grad")
    return loss.value, g


def sse_nn_train(plan, x, t, steps, batch, lr, seed=0, stream=None):
    """Adam training; returns the loss of every step."""
    import numpy as np
    n, H, W = x.shape
    losses = np.zeros(steps, dtype=np.float64)
    _check(load().sse_nn_train(plan, _ptr(x), _ptr(t), n, H, W, steps, batch, lr, seed,
                               losses.ctypes.data, _stream(stream)), "sse_nn_train")
    return losses


def soft_destroy(plan):
    if plan:
        load().soft_destroy(plan)


def soft_plan_points(plan, i=0):
    return load().soft_plan_points(plan, i)


def soft_plan_count(plan):
    return load().soft_plan_count(plan)


def soft_last_launches(plan):
    return load().soft_last_launches(plan)


class Plan:
    """Owns a plan handle (destroyed on close / garbage collection)."""

    def __init__(self, handle):
        self.h = handle

    def close(self):
        if self.h:
            soft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
