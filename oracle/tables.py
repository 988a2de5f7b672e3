"""Oracle: grid, momentum table, complex contour and the finite-difference
absorbing matrix C, in plain FP64 numpy.

This module is TEST INFRASTRUCTURE.  It is the slow, obviously-correct CPU
statement of what the GPU library computes; only ``tests/``, the smoke check
and the CPU-baseline leg of the benchmark may import it.  It shares no code
with the CUDA path.

Every function cites the passage of Serov & Sergeeva, "Solution of the
Schroedinger equation using exterior complex scaling and fast Fourier
transform" (arXiv:1505.06707) that it follows.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid", "kgrid", "midpoints", "q_contour", "z_contour", "soft_coulomb",
    "c_tridiag", "ks_tridiag", "kfd_tridiag", "dense_from_tridiag",
    "strip_block", "field_E",
]

# contour kinds; CAP and TFAP are the comparison absorbers of Sec. IV: the
# contour stays real (q = 1, z = x) and a complex potential absorbs instead
SHARP, SECS, TFECS, CAP, TFAP = 0, 1, 2, 3, 4

# c of Eq. yTFAP (the value the paper quotes)
TFAP_C = 2.622057


def grid(n: int, a: float, b: float):
    """Half-shifted uniform grid x_i = a + h(i - 1/2), i = 1..N, h = (b-a)/N
    (Sec. II, Eq. DVRgrid).  Returned 0-based: x[j] = a + h(j + 1/2)."""
    h = (b - a) / n
    return a + h * (np.arange(n, dtype=np.float64) + 0.5), h


def kgrid(n: int, a: float, b: float):
    """Fourier momenta k_n (Sec. II, the table under Eq. FFTbasis):
    k = 2 pi (n-1)/(b-a) for n <= N/2, -2 pi (N+1-n)/(b-a) otherwise.
    0-based index m = n - 1; the index m = N/2 (Nyquist) is negative."""
    L = b - a
    m = np.arange(n, dtype=np.float64)
    return np.where(m < n // 2, 2.0 * np.pi * m / L, -2.0 * np.pi * (n - m) / L)


def midpoints(n: int, a: float, b: float):
    """x_{i+1/2} for 0-based i = 0..N-1, i.e. a + h(i+1); the last one is b,
    which the periodic grid identifies with a."""
    h = (b - a) / n
    return a + h * (np.arange(n, dtype=np.float64) + 1.0)


def _tfecs_ytilde(s, alpha):
    # Sec. IV, Eq. qTFECS: ytilde(s) = alpha[(1-s)^-2 - (1+s)^-2 - 4s]
    return alpha * (1.0 / (1.0 - s) ** 2 - 1.0 / (1.0 + s) ** 2 - 4.0 * s)


def q_contour(x, kind: int, R0: float, rmax: float, theta: float = 0.0,
              alpha: float = 0.5):
    """Contour derivative q(x) (Sec. II, Eq. ECSintdef; Sec. IV).

    SHARP: q = 1 for |x| <= R0, exp(i theta) beyond (Sec. IV, sharp rotation;
           the point |x| = R0 itself is read as unscaled).
    SECS:  q = exp[i theta (|x|-R0)/dx_CS], dx_CS = rmax - R0: Eq. qSECS with
           its final angle pi/4 made a parameter (theta = pi/4 is the paper's
           contour; the laser batch uses theta = 0.5, see the workloads).
    TFECS: q = sqrt(1 + i ytilde(s)), s = (|x|-R0)/dx_CS (Eq. qTFECS).
    TFECS is infinite at |x| = rmax; callers that need 1/q there use
    ``inv_q``."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    q = np.ones(x.shape, dtype=np.complex128)
    out = ax > R0
    if kind == SHARP:
        q[out] = np.exp(1j * theta)
    elif kind == SECS:
        q[out] = np.exp(1j * theta * (ax[out] - R0) / (rmax - R0))
    elif kind == TFECS:
        s = (ax[out] - R0) / (rmax - R0)
        with np.errstate(divide="ignore", invalid="ignore"):
            q[out] = np.sqrt(1.0 + 1j * _tfecs_ytilde(s, alpha))
    elif kind in (CAP, TFAP):
        pass                                # unscaled: the absorber is a potential
    else:
        raise ValueError("unknown contour kind")
    return q


def inv_q(x, kind, R0, rmax, theta=0.0, alpha=0.5):
    """1/q(x), with the TFECS limit 1/q -> 0 at |x| = rmax."""
    x = np.asarray(x, dtype=np.float64)
    q = q_contour(x, kind, R0, rmax, theta, alpha)
    r = np.zeros_like(q)
    fin = np.isfinite(q)
    r[fin] = 1.0 / q[fin]
    return r


def z_contour(x, kind: int, R0: float, rmax: float, theta: float = 0.0,
              alpha: float = 0.5):
    """Complex coordinate z(x) = int_0^x q (Sec. II, Eq. ECSintdef).

    SHARP and SECS have closed forms; TFECS is integrated by adaptive
    quadrature (a library primitive)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    sg = np.sign(x)
    z = x.astype(np.complex128)
    out = ax > R0
    d = ax[out] - R0
    if kind == SHARP:
        z[out] = sg[out] * (R0 + np.exp(1j * theta) * d)
    elif kind == SECS:
        if theta == 0.0:                    # q = 1: no scaling
            z[out] = x[out]
        else:
            c = 1j * theta / (rmax - R0)
            z[out] = sg[out] * (R0 + (np.exp(c * d) - 1.0) / c)
    elif kind == TFECS:
        from scipy.integrate import quad
        vals = []
        for dd in d:
            f_re = lambda t: np.real(q_contour(np.array([R0 + t]), TFECS, R0, rmax, 0.0, alpha)[0])
            f_im = lambda t: np.imag(q_contour(np.array([R0 + t]), TFECS, R0, rmax, 0.0, alpha)[0])
            re = quad(f_re, 0.0, dd, limit=200, epsabs=1e-14, epsrel=1e-13)[0]
            im = quad(f_im, 0.0, dd, limit=200, epsabs=1e-14, epsrel=1e-13)[0]
            vals.append(R0 + re + 1j * im)
        z[out] = sg[out] * np.array(vals, dtype=np.complex128)
    elif kind in (CAP, TFAP):
        pass
    else:
        raise ValueError("unknown contour kind")
    return z


def tfap_y(s):
    """y(s) of Eq. yTFAP: [a s - b s^3 + 4/(1-s)^2 - 4/(1+s)^2] / c^2 with
    a = c^3 - 16, b = c^3 - 17."""
    c = TFAP_C
    a, b = c ** 3 - 16.0, c ** 3 - 17.0
    s = np.asarray(s, dtype=np.float64)
    return (a * s - b * s ** 3 + 4.0 / (1.0 - s) ** 2 - 4.0 / (1.0 + s) ** 2) / (c * c)


def absorbing_potential(x, kind: int, R0: float, rmax: float, theta: float = np.pi / 4,
                        e_cap: float = 2.0, kmin: float = 0.25):
    """Complex absorbing potential U_a(x) of the comparison absorbers of
    Sec. IV, zero for |x| <= R0 (= r_s), dx_CS = rmax - R0:
      CAP:  U_a = E_CAP [1 - q(x)^2] with q of Eq. qSECS (final angle theta)
            -- Eq. CAP_via_q, the CAP equivalent to ECS at energy E_CAP;
      TFAP: U_a = -i (k_min^2 / 2) y((|x| - r_s)/dx_CS)  -- Eqs. TFAP, yTFAP.
    Other kinds have none (zeros)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    u = np.zeros(x.shape, dtype=np.complex128)
    out = ax > R0
    if kind == CAP:
        q = np.exp(1j * theta * (ax[out] - R0) / (rmax - R0))
        u[out] = e_cap * (1.0 - q * q)
    elif kind == TFAP:
        u[out] = -0.5j * kmin * kmin * tfap_y((ax[out] - R0) / (rmax - R0))
    return u


def soft_coulomb(z_list, a2: float, charge: float = 1.0):
    """U(z) = -Z / sqrt(sum_d z_d^2 + a^2) evaluated at the complex
    coordinate(s) (Sec. II: the potential is taken at z(x)).  Principal
    square root."""
    s = np.zeros(np.broadcast(*z_list).shape, dtype=np.complex128) + a2
    for z in z_list:
        s = s + np.asarray(z, dtype=np.complex128) ** 2
    return -charge / np.sqrt(s)


def ks_tridiag(n, a, b, kind, R0, theta=0.0, alpha=0.5):
    """Three-point K_s of Sec. II, Eq. Ks_FD, with periodic wrap.

    Row i: [K_s psi]_i = -(1/2h) q_i^{-1/2} [ (q_{i+1}^{-1/2} psi_{i+1}
    - q_i^{-1/2} psi_i)/(q_{i+1/2} h) - (q_i^{-1/2} psi_i - q_{i-1}^{-1/2}
    psi_{i-1})/(q_{i-1/2} h) ].  Returns (sub, diag, sup): sub[i] multiplies
    psi_{i-1}, sup[i] multiplies psi_{i+1} (indices mod N)."""
    rmax = b  # the contour is defined on the symmetric box |x| <= b
    x, h = grid(n, a, b)
    xm = midpoints(n, a, b)                   # x_{i+1/2}
    qi = q_contour(x, kind, R0, rmax, theta, alpha)
    qhm = qi ** -0.5                          # q_i^{-1/2}, principal branch
    iq_p = inv_q(xm, kind, R0, rmax, theta, alpha)          # 1/q_{i+1/2}
    iq_m = np.roll(iq_p, 1)                                  # 1/q_{i-1/2}
    qh_p = np.roll(qhm, -1)                                  # q_{i+1}^{-1/2}
    qh_m = np.roll(qhm, 1)                                   # q_{i-1}^{-1/2}
    c = -0.5 / (h * h)
    sup = c * qhm * qh_p * iq_p
    sub = c * qhm * qh_m * iq_m
    diag = -c * qhm * qhm * (iq_p + iq_m)
    return sub, diag, sup


def kfd_tridiag(n, a, b):
    """Free three-point kinetic K_FD of Sec. II, Eq. K_FD (periodic)."""
    h = (b - a) / n
    c = -0.5 / (h * h)
    sub = np.full(n, c, dtype=np.complex128)
    sup = np.full(n, c, dtype=np.complex128)
    diag = np.full(n, -2.0 * c, dtype=np.complex128)
    return sub, diag, sup


def c_tridiag(n, a, b, kind, R0, theta=0.0, alpha=0.5):
    """Absorbing matrix C = K_s - K_FD (Sec. II, Eq. C_FD): complex symmetric,
    tridiagonal, periodic; zero wherever q = 1 on a row and its neighbours."""
    s1, d1, u1 = ks_tridiag(n, a, b, kind, R0, theta, alpha)
    s0, d0, u0 = kfd_tridiag(n, a, b)
    return s1 - s0, d1 - d0, u1 - u0


def dense_from_tridiag(sub, diag, sup):
    """Dense N x N matrix of a periodic tridiagonal (tests, tiny N)."""
    n = len(diag)
    M = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        M[i, i] += diag[i]
        M[i, (i - 1) % n] += sub[i]
        M[i, (i + 1) % n] += sup[i]
    return M


def strip_block(sub, diag, sup):
    """Rows on which C is non-zero, as a set of indices (used by tests to
    check that the GPU's strip-only solve covers every coupled row)."""
    nz = (np.abs(sub) + np.abs(diag) + np.abs(sup)) > 0
    return np.nonzero(nz)[0]


def field_E(t, E0, omega, ncycles=4.0):
    """Laser field E(t) = E0 sin^2(pi t / T) sin(omega t), T = ncycles 2 pi/omega,
    zero outside [0, T] (the pulse of the batched laser workload; the paper
    itself only requires U(x, t) at t + tau/2, Sec. II under Eq. SSFFT)."""
    T = ncycles * 2.0 * np.pi / omega
    t = np.asarray(t, dtype=np.float64)
    e = E0 * np.sin(np.pi * t / T) ** 2 * np.sin(omega * t)
    return np.where((t >= 0) & (t <= T), e, 0.0)
