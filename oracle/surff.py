"""Oracle for the amplitude extraction the paper's test uses (Sec. I and
Sec. IV: t&E-SURFF): momentum amplitudes of the outgoing part of the wave
function from the probability-amplitude flux through the boundary x = +-R
of the unscaled region up to t_max (t-SURFF), plus the part still inside at
t_max from the stationary ECS equation with right-hand side psi(t_max)
(E-SURFF, the SSE of Sec. III).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The paper cites the formulas (Serov 2013) without printing them; they are
written out here from the free-particle dynamics beyond R (U = 0 there, as
in the paper's test).  With plane waves chi_k(x, t) = (2 pi)^-1/2
e^{i k x - i E t}, E = k^2/2, the amplitude A(k) = <chi_k(t)|psi(t)> of a
free packet is constant in time, and for k > 0 it is the limit of the
overlap over x > R.  Its time derivative is a surface term, so

  A(k) = -(i/2) (2 pi)^-1/2 e^{-ikR} [ int_0^T e^{iEt} g_R(t) dt
                                        + i e^{iET} D_k phi_E(R) ],
  g_R(t) = psi'(R, t) + i k psi(R, t),   D_k phi = phi' + i k phi,
  (E - H) phi_E = psi(T)

(the second term is the time integral from T to infinity: int_T^inf
e^{iEt} e^{-iH(t-T)} dt = i e^{iET} (E - H)^-1 with outgoing conditions,
which the ECS resolvent provides).  For k < 0 the left boundary x = -R
gives the same with the opposite overall sign and e^{+ikR}.  psi and psi'
at +-R come from the trigonometric interpolant of the grid function (the
FFT representation of Sec. II); the time integral is Simpson's rule or the
Filon-Simpson rule for e^{iEt} times a quadratic on each pair of steps
(Sec. IV, the closing comparison of the two rules)."""
from __future__ import annotations

import math

import numpy as np


def surface_weights(x, k, R):
    """Rows w such that w @ psi gives psi(R), psi'(R), psi(-R), psi'(-R) for
    the trigonometric interpolant psi(x) = (1/N) sum_m c_m e^{i k_m (x - x_0)},
    c = FFT(psi) (numpy's e^{-2 pi i m j/N})."""
    n = len(x)
    j = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(np.arange(n), j) / n)     # c = F psi
    rows = []
    for xs in (R, -R):
        e = np.exp(1j * k * (xs - x[0])) / n
        rows.append(e @ F)
        rows.append((1j * k * e) @ F)
    return np.array(rows)


def surface_values(psi, x, k, R):
    """psi(R), psi'(R), psi(-R), psi'(-R) through numpy's FFT (the same
    interpolant as ``surface_weights``)."""
    n = len(x)
    c = np.fft.fft(psi)
    out = []
    for xs in (R, -R):
        e = np.exp(1j * k * (xs - x[0])) / n
        out.append(np.sum(c * e))
        out.append(np.sum(c * 1j * k * e))
    return np.array(out)


def record(problem, psi0, nsteps, t0=0.0, field=None):
    """Propagate with the oracle step one step at a time and record the
    surface values at t0 + s tau, s = 0 .. nsteps (rows: psi(R), psi'(R),
    psi(-R), psi'(-R)), with R the problem's R0.  Returns (samples, psi(T))."""
    R = problem.R0
    out = np.zeros((nsteps + 1, 4), dtype=np.complex128)
    psi = np.asarray(psi0, dtype=np.complex128)
    out[0] = surface_values(psi, problem.x, problem.k, R)
    for s in range(nsteps):
        psi = problem.step(psi, 1, t0=t0 + s * problem.dt, field=field)
        out[s + 1] = surface_values(psi, problem.x, problem.k, R)
    return out, psi


def _panel_moments(th, tau):
    """int_{-tau}^{tau} e^{i w u} u^p du for p = 0, 1, 2, with th = w tau
    (series for small |th|)."""
    if abs(th) < 1e-3:
        t2 = th * th
        m0 = 2 * tau * (1 - t2 / 6 + t2 * t2 / 120)
        m1 = 2j * tau * tau * th * (1.0 / 3 - t2 / 30)
        m2 = 2 * tau ** 3 * (1.0 / 3 - t2 / 10 + t2 * t2 / 168)
        return m0, m1, m2
    s, c = math.sin(th), math.cos(th)
    w = th / tau
    m0 = 2 * s / w
    m1 = 2j * (s - th * c) / (w * w)
    m2 = 2 * ((th * th - 2) * s + 2 * th * c) / w ** 3
    return m0, m1, m2


def time_integral(g, tau, omega, t0=0.0, rule="simpson"):
    """int_{t0}^{t0 + M tau} e^{i omega t} g(t) dt from samples g_s = g(t0 + s tau),
    M even.  simpson: Simpson's rule on the whole integrand; filon: on each
    pair of steps g is replaced by its quadratic interpolant and the product
    with e^{i omega t} integrated exactly (Filon-Simpson)."""
    g = np.asarray(g)
    M = len(g) - 1
    if M % 2:
        raise ValueError("an even number of steps")
    t = t0 + tau * np.arange(M + 1)
    if rule == "simpson":
        f = np.exp(1j * omega * t) * g
        return tau / 3 * (f[0] + f[-1] + 4 * np.sum(f[1:-1:2]) + 2 * np.sum(f[2:-1:2]))
    if rule != "filon":
        raise ValueError(rule)
    m0, m1, m2 = _panel_moments(omega * tau, tau)
    acc = 0.0 + 0.0j
    for j in range(0, M, 2):
        g0, g1, g2 = g[j], g[j + 1], g[j + 2]
        a = g1
        b = (g2 - g0) / (2 * tau)
        c = (g2 - 2 * g1 + g0) / (2 * tau * tau)
        acc += np.exp(1j * omega * t[j + 1]) * (a * m0 + b * m1 + c * m2)
    return acc


def amplitudes(samples, phiA, E, R, tau, t0=0.0, rule="simpson", weights=None):
    """A(+k) and A(-k), k = sqrt(2E), from the surface samples (rows as in
    ``record``, times t0 + s tau) and the solution phiA of A phiA = psi(T)
    with the matrix A = H - E of Sec. III (Eq. linsys), so that
    phi_E = -phiA; phiA is given by its four surface values, or as a grid
    function together with ``weights`` (surface_weights).  Returns
    (A(+k), A(-k))."""
    k = math.sqrt(2 * E)
    T = t0 + tau * (len(samples) - 1)
    ps = -(weights @ phiA if weights is not None else np.asarray(phiA))
    pre = (2 * math.pi) ** -0.5
    out = []
    for kk, col, sgn in ((k, 0, -1.0), (-k, 2, 1.0)):
        xs = R if col == 0 else -R
        g = samples[:, col + 1] + 1j * kk * samples[:, col]
        It = time_integral(g, tau, E, t0, rule)
        De = ps[col + 1] + 1j * kk * ps[col]
        out.append(sgn * 0.5j * pre * np.exp(-1j * kk * xs) * (It + 1j * np.exp(1j * E * T) * De))
    return out[0], out[1]


def a_teor(k, v0):
    """Eq. Ateor: pi^-1/4 exp[-(k - v0)^2 / 2], the spectrum of the packet of
    Eq. psi0."""
    return math.pi ** -0.25 * np.exp(-(np.asarray(k) - v0) ** 2 / 2)
