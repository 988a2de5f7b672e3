"""Seeded synthetic workloads: problem parameters and initial states.

This module holds NO arithmetic of the method: it draws random parameters
(numpy PCG64 from ``SeedSequence([1505, workload, item])``) and evaluates
Gaussian packets on the half-shifted grid.  Both the GPU library's tests and
benchmark and the oracle consume what it returns; neither side imports the
other.

Workloads (all lengths in atomic units):
  W1  1D single instance: N=1024 on [-200,200], soft-Coulomb a^2=2, sharp ECS
      at R0=150 with theta=0.5, Gaussian x0=0 sigma=5 k0=1 with a seeded global
      phase; dt=0.05, 2000 steps.
  W2  1D batch in a laser pulse: 4096 instances, N drawn from {2048..16384},
      box [-8N/1024, 8N/1024] (h=1/64), R0 = 0.75 of the half-width, smooth
      (SECS) contour reaching theta=0.5 at the box edge, a^2=2 (the sharp
      contour makes the scheme unstable on this grid: spectral radius 1.046
      per step); pulse E0 sin^2(pi t/T) sin(omega t), omega=0.057, 4 cycles,
      E0 ~ U[0.01, 0.1]; dt=0.02, 22046 steps to the pulse end.  Initial state:
      a seeded real-centred Gaussian (sigma ~ U[1,2]) with a seeded phase.
  W3  2D single instance: 2048^2 on [-200,200]^2, U=-1/sqrt(x^2+y^2+1), sharp
      ECS on both axes R0=150 theta=0.4; sum of 4 seeded Gaussians (centres in
      [-50,50]^2, sigma ~ U[3,8], |k| <= 1.5, phases); dt=0.02, 10000 steps.
  W4  Stationary solves: 1024^2 on the W3 box and contour; source chi a
      Gaussian (sigma 4, seeded centre in [-10,10]^2, seeded phase); 64
      energies ~ U[0.05, 2.0] sorted; tolerance 1e-8.  The linear system is
      A psi = f with f = -chi (A = H - E).
  W6  3D single instance: 256^3 on [-40,40]^3 (h = 0.3125),
      U=-1/sqrt(x^2+y^2+z^2+1), sharp ECS on every axis R0=30 theta=0.4;
      sum of 4 seeded Gaussians (centres within a quarter of the half-width,
      sigma ~ U[0.08, 0.15] of the half-width, |k| <= 1.5, phases); dt=0.02.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 1505


def rng(workload: int, item: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED, workload, item])))


def half_shifted_grid(n, a, b):
    """x_j = a + h (j + 1/2), h = (b - a)/n."""
    h = (b - a) / n
    return a + h * (np.arange(n, dtype=np.float64) + 0.5), h


def gaussian(x, x0, sigma, k0, phase):
    """(pi sigma^2)^{-1/4} exp(-(x-x0)^2/(2 sigma^2) + i k0 x + i phase)."""
    return ((math.pi * sigma * sigma) ** -0.25
            * np.exp(-(x - x0) ** 2 / (2 * sigma * sigma) + 1j * k0 * x + 1j * phase))


def normalise(psi, dvol):
    return psi / math.sqrt(dvol * float(np.sum(np.abs(psi) ** 2)))


# ---------------------------------------------------------------- W1 ------
def w1(n=1024, a=-200.0, b=200.0):
    g = rng(1, 0)
    phase = g.uniform(0.0, 2 * math.pi)
    x, h = half_shifted_grid(n, a, b)
    psi0 = gaussian(x, 0.0, 5.0, 1.0, phase)
    return dict(n=n, a=a, b=b, R0=150.0, theta=0.5, a2=2.0, dt=0.05, nsteps=2000,
                sigma=5.0, x0=0.0, k0=1.0, phase=phase, psi0=psi0)


# ---------------------------------------------------------------- W2 ------
W2_SIZES = (2048, 4096, 8192, 16384)
W2_OMEGA = 0.057
W2_NCYC = 4.0
W2_DT = 0.02
W2_CONTOUR = 1          # SECS (smooth) with final angle theta


def w2_nsteps():
    T = W2_NCYC * 2 * math.pi / W2_OMEGA
    return int(round(T / W2_DT))


def w2_instance(j: int):
    """Parameters and initial state of instance j of the laser batch."""
    g = rng(2, j)
    n = int(g.choice(W2_SIZES))
    hw = 8.0 * n / 1024.0
    E0 = g.uniform(0.01, 0.1)
    sigma = g.uniform(1.0, 2.0)
    phase = g.uniform(0.0, 2 * math.pi)
    x, h = half_shifted_grid(n, -hw, hw)
    psi0 = normalise(gaussian(x, 0.0, sigma, 0.0, phase), h)
    return dict(n=n, a=-hw, b=hw, R0=0.75 * hw, theta=0.5, contour=W2_CONTOUR, a2=2.0, dt=W2_DT,
                E0=E0, omega=W2_OMEGA, ncyc=W2_NCYC, psi0=psi0)


def w2_sizes(count=4096):
    return [int(rng(2, j).choice(W2_SIZES)) for j in range(count)]


# ---------------------------------------------------------------- W3 ------
def w3(n=2048, box=(-200.0, 200.0, -200.0, 200.0), ngauss=4):
    g = rng(3, 0)
    x, hx = half_shifted_grid(n, box[0], box[1])
    y, hy = half_shifted_grid(n, box[2], box[3])
    psi = np.zeros((n, n), dtype=np.complex128)
    for _ in range(ngauss):
        cx, cy = g.uniform(-50, 50, size=2)
        sg = g.uniform(3.0, 8.0)
        kr = 1.5 * math.sqrt(g.uniform(0, 1))
        ka = g.uniform(0, 2 * math.pi)
        ph = g.uniform(0, 2 * math.pi)
        gx = gaussian(x, cx, sg, kr * math.cos(ka), ph)
        gy = gaussian(y, cy, sg, kr * math.sin(ka), 0.0)
        psi += gy[:, None] * gx[None, :]
    psi = normalise(psi, hx * hy)
    return dict(nx=n, ny=n, box=box, R0=150.0, theta=0.4, a2=1.0, dt=0.02, nsteps=10000,
                psi0=psi)


# ---------------------------------------------------------------- W4 ------
def w4(n=1024, box=(-200.0, 200.0, -200.0, 200.0), n_energies=64):
    g = rng(4, 0)
    cx, cy = g.uniform(-10, 10, size=2)
    ph = g.uniform(0, 2 * math.pi)
    E = np.sort(g.uniform(0.05, 2.0, size=n_energies))
    x, hx = half_shifted_grid(n, box[0], box[1])
    y, hy = half_shifted_grid(n, box[2], box[3])
    chi = gaussian(y, cy, 4.0, 0.0, 0.0)[:, None] * gaussian(x, cx, 4.0, 0.0, ph)[None, :]
    return dict(nx=n, ny=n, box=box, R0=150.0, theta=0.4, a2=1.0, E=E, tol=1e-8,
                chi=chi, f=-chi)


# ---------------------------------------------------------------- W6 ------
def w6_state(n, box, seed=0, ngauss=4, noise=0.0):
    """Sum of ngauss seeded 3D Gaussians on the [nz][ny][nx] grid of box
    (ax, bx, ay, by, az, bz), normalised; `noise` adds that fraction of
    seeded complex white noise (it reaches every mode, the strips included)."""
    g = rng(6, seed)
    ax = [half_shifted_grid(n[d], box[2 * d], box[2 * d + 1]) for d in range(3)]
    half = min(box[2 * d + 1] for d in range(3))
    psi = np.zeros((n[2], n[1], n[0]), dtype=np.complex128)
    for _ in range(ngauss):
        c = [g.uniform(-0.25, 0.25) * box[2 * d + 1] for d in range(3)]
        sg = g.uniform(0.08, 0.15) * half
        k = g.uniform(-1.0, 1.0, size=3)
        k *= 1.5 * math.sqrt(g.uniform(0, 1)) / max(1e-12, float(np.linalg.norm(k)))
        ph = g.uniform(0, 2 * math.pi)
        f = [gaussian(ax[d][0], c[d], sg, k[d], ph if d == 0 else 0.0) for d in range(3)]
        psi += f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    if noise:
        psi += noise * float(np.abs(psi).max()) * (g.standard_normal(psi.shape)
                                                  + 1j * g.standard_normal(psi.shape))
    return normalise(psi, ax[0][1] * ax[1][1] * ax[2][1])


def w6(n=256, half=40.0):
    """The 3D benchmark workload (parameters; the state from w6_state)."""
    return dict(n=(n, n, n), box=(-half, half) * 3, R0=30.0, theta=0.4, kind=0, a2=1.0,
                dt=0.02)
