"""Oracle time propagation: ctypes front end of ``soft_oracle.c`` plus the
per-problem tables it needs (built here from ``oracle.tables``).

TEST INFRASTRUCTURE (see ``oracle/__init__``)."""
from __future__ import annotations

import ctypes as C
import numpy as np

from . import tables as T
from .build import build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_fft.argtypes = [P, C.c_int, C.c_int]
        _lib.orc_cyclic_solve.argtypes = [C.c_int, P, P, P, P, P]
        _lib.orc_cyclic_solve.restype = C.c_int
        _lib.orc_step1d.argtypes = [C.c_int, C.c_long, P, P, P, P, P, P, P,
                                    C.c_double, C.c_double, C.c_int, C.c_double,
                                    C.c_double, C.c_double]
        _lib.orc_step1d.restype = C.c_int
        _lib.orc_step1d_batch.argtypes = [C.c_int, P, P, C.c_long, P, P, P, P, P, P,
                                          P, P, P, P, P, P, P]
        _lib.orc_step1d_batch.restype = C.c_int
        _lib.orc_step2d.argtypes = [C.c_int, C.c_int, C.c_long, P, P, P, P, P, P, P,
                                    P, P, P, C.c_double]
        _lib.orc_step2d.restype = C.c_int
        _lib.orc_step3d.argtypes = [C.c_int, C.c_int, C.c_int, C.c_long, P, P, P, P, P,
                                    P, P, P, C.c_double]
        _lib.orc_step3d.restype = C.c_int
        _lib.orc_num_threads.restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def fft(a, sign=-1):
    """Radix-2 DFT of the oracle (unnormalised); sign -1 = e^{-i...}."""
    a = np.ascontiguousarray(a, dtype=np.complex128).copy()
    lib().orc_fft(_p(a), len(a), sign)
    return a


def cyclic_solve(sub, diag, sup, r):
    """Periodic tridiagonal solve (Sherman-Morrison + pivoted elimination)."""
    n = len(diag)
    x = np.ascontiguousarray(r, dtype=np.complex128).copy()
    work = np.zeros(16 * n, dtype=np.complex128)
    s = np.ascontiguousarray(sub, dtype=np.complex128)
    d = np.ascontiguousarray(diag, dtype=np.complex128)
    u = np.ascontiguousarray(sup, dtype=np.complex128)
    if lib().orc_cyclic_solve(n, _p(s), _p(d), _p(u), _p(x), _p(work)):
        raise FloatingPointError("singular tridiagonal system")
    return x


class Problem1D:
    """All per-point tables of one 1D instance (Sec. II).

    kind/R0/theta/alpha choose the contour q(x); the potential is the
    soft-Coulomb U(z) = -Z/sqrt(z^2 + a2) at z(x) (Sec. II, Eq. psi_zx and
    the text after it); ``xc`` is the dipole coordinate clamp(x, -R0, R0)
    multiplying the laser field (a reading: the field is switched off inside
    the scaled strips, where continuing x to z would make it grow)."""

    def __init__(self, n, a, b, R0, theta=0.5, kind=T.SHARP, alpha=0.5, a2=2.0,
                 charge=1.0, dt=0.05, potential=True, e_cap=2.0, kmin=0.25):
        self.n, self.a, self.b, self.R0, self.theta = n, a, b, R0, theta
        self.kind, self.alpha, self.dt = kind, alpha, dt
        self.x, self.h = T.grid(n, a, b)
        self.k = T.kgrid(n, a, b)
        self.q = T.q_contour(self.x, kind, R0, b, theta, alpha)
        self.z = T.z_contour(self.x, kind, R0, b, theta, alpha)
        if potential:
            self.U0 = T.soft_coulomb([self.z], a2, charge)
        else:
            self.U0 = np.zeros(n, dtype=np.complex128)
        # CAP / TFAP comparison absorbers (Sec. IV): a complex potential
        self.U0 = self.U0 + T.absorbing_potential(self.x, kind, R0, b, theta, e_cap, kmin)
        self.xc = np.clip(self.x, -R0, R0)
        self.Cs, self.Cd, self.Cu = T.c_tridiag(n, a, b, kind, R0, theta, alpha)

    def step(self, psi, nsteps, t0=0.0, field=None):
        """nsteps literal steps; field = (E0, omega, ncycles) or None."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
        k = np.ascontiguousarray(self.k)
        U0 = np.ascontiguousarray(self.U0)
        xc = np.ascontiguousarray(self.xc)
        hf = 0 if field is None else 1
        E0, om, nc = (0.0, 1.0, 1.0) if field is None else field
        rc = lib().orc_step1d(self.n, int(nsteps), _p(psi), _p(k), _p(U0), _p(xc),
                              _p(self.Cs), _p(self.Cd), _p(self.Cu), float(self.dt),
                              float(t0), hf, float(E0), float(om), float(nc))
        if rc:
            raise FloatingPointError("oracle step failed (%d)" % rc)
        return psi


def step_batch(problems, psis, nsteps, t0s=None, fields=None):
    """Independent 1D instances side by side (OpenMP over instances)."""
    cnt = len(problems)
    ns = np.array([p.n for p in problems], dtype=np.int32)
    off = np.zeros(cnt, dtype=np.int64)
    off[1:] = np.cumsum(ns[:-1])
    cat = lambda f: np.ascontiguousarray(np.concatenate([f(p) for p in problems]))
    psi = np.ascontiguousarray(np.concatenate(psis).astype(np.complex128))
    k, U0, xc = cat(lambda p: p.k), cat(lambda p: p.U0), cat(lambda p: p.xc)
    Cs, Cd, Cu = cat(lambda p: p.Cs), cat(lambda p: p.Cd), cat(lambda p: p.Cu)
    tau = np.array([p.dt for p in problems], dtype=np.float64)
    t0 = np.zeros(cnt) if t0s is None else np.asarray(t0s, dtype=np.float64)
    if fields is None:
        fields = [None] * cnt
    hf = np.array([0 if f is None else 1 for f in fields], dtype=np.int32)
    E0 = np.array([0.0 if f is None else f[0] for f in fields])
    om = np.array([1.0 if f is None else f[1] for f in fields])
    nc = np.array([1.0 if f is None else f[2] for f in fields])
    rc = lib().orc_step1d_batch(cnt, _p(ns), _p(off), int(nsteps), _p(psi), _p(k), _p(U0),
                                _p(xc), _p(Cs), _p(Cd), _p(Cu), _p(tau), _p(t0), _p(hf),
                                _p(E0), _p(om), _p(nc))
    if rc:
        raise FloatingPointError("oracle batch step failed")
    return [psi[o:o + n].copy() for o, n in zip(off, ns)]


class Problem2D:
    """2D instance on [ax,bx] x [ay,by], psi stored [ny][nx] (x fastest).
    Same contour kind on both axes; U = -Z/sqrt(z_x^2 + z_y^2 + a2)."""

    def __init__(self, nx, ny, box, R0, theta=0.4, kind=T.SHARP, alpha=0.5, a2=1.0,
                 charge=1.0, dt=0.02, potential=True, e_cap=2.0, kmin=0.25):
        ax, bx, ay, by = box
        self.nx, self.ny, self.box, self.dt = nx, ny, box, dt
        self.x, self.hx = T.grid(nx, ax, bx)
        self.y, self.hy = T.grid(ny, ay, by)
        self.kx, self.ky = T.kgrid(nx, ax, bx), T.kgrid(ny, ay, by)
        zx = T.z_contour(self.x, kind, R0, bx, theta, alpha)
        zy = T.z_contour(self.y, kind, R0, by, theta, alpha)
        if potential:
            self.U = T.soft_coulomb([zx[None, :], zy[:, None]], a2, charge)
        else:
            self.U = np.zeros((ny, nx), dtype=np.complex128)
        # comparison absorbers: U_a(x) + U_a(y)
        self.U = (self.U + T.absorbing_potential(self.x, kind, R0, bx, theta, e_cap, kmin)[None, :]
                  + T.absorbing_potential(self.y, kind, R0, by, theta, e_cap, kmin)[:, None])
        self.U = np.ascontiguousarray(self.U, dtype=np.complex128)
        self.Cx = T.c_tridiag(nx, ax, bx, kind, R0, theta, alpha)
        self.Cy = T.c_tridiag(ny, ay, by, kind, R0, theta, alpha)

    def step(self, psi, nsteps):
        psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
        cx = [np.ascontiguousarray(c) for c in self.Cx]
        cy = [np.ascontiguousarray(c) for c in self.Cy]
        rc = lib().orc_step2d(self.nx, self.ny, int(nsteps), _p(psi), _p(self.kx),
                              _p(self.ky), _p(self.U), _p(cx[0]), _p(cx[1]), _p(cx[2]),
                              _p(cy[0]), _p(cy[1]), _p(cy[2]), float(self.dt))
        if rc:
            raise FloatingPointError("oracle 2D step failed")
        return psi


class Problem3D:
    """3D instance on box = (ax, bx, ay, by, az, bz), psi stored [nz][ny][nx]
    (x fastest).  Same contour kind on the three axes;
    U = -Z/sqrt(z_x^2 + z_y^2 + z_z^2 + a2) plus the axes' absorber terms."""

    def __init__(self, n, box, R0, theta=0.4, kind=T.SHARP, alpha=0.5, a2=1.0,
                 charge=1.0, dt=0.02, potential=True, e_cap=2.0, kmin=0.25):
        self.n, self.box, self.dt = tuple(n), tuple(box), dt
        self.x, self.k, z, ua, self.C = [], [], [], [], []
        for d in range(3):
            a, b = box[2 * d], box[2 * d + 1]
            xd, _ = T.grid(n[d], a, b)
            self.x.append(xd)
            self.k.append(T.kgrid(n[d], a, b))
            z.append(T.z_contour(xd, kind, R0, b, theta, alpha))
            ua.append(T.absorbing_potential(xd, kind, R0, b, theta, e_cap, kmin))
            self.C.append(T.c_tridiag(n[d], a, b, kind, R0, theta, alpha))
        zx, zy, zz = z[0][None, None, :], z[1][None, :, None], z[2][:, None, None]
        if potential:
            U = T.soft_coulomb([zx, zy, zz], a2, charge)
        else:
            U = np.zeros((n[2], n[1], n[0]), dtype=np.complex128)
        U = U + ua[0][None, None, :] + ua[1][None, :, None] + ua[2][:, None, None]
        self.U = np.ascontiguousarray(np.broadcast_to(U, (n[2], n[1], n[0])), dtype=np.complex128)

    def step(self, psi, nsteps):
        psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
        cs, cd, cu = (np.ascontiguousarray(np.concatenate([c[i] for c in self.C]))
                      for i in range(3))
        k = [np.ascontiguousarray(kk) for kk in self.k]
        U = np.ascontiguousarray(self.U)
        rc = lib().orc_step3d(self.n[0], self.n[1], self.n[2], int(nsteps), _p(psi),
                              _p(k[0]), _p(k[1]), _p(k[2]), _p(U), _p(cs), _p(cd), _p(cu),
                              float(self.dt))
        if rc:
            raise FloatingPointError("oracle 3D step failed")
        return psi


def num_threads():
    return int(lib().orc_num_threads())
