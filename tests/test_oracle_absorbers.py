"""Pins of the oracle's comparison absorbers and of its stationary solver on
the paper's own test (Sec. IV): the linear CAP of Eq. CAP_via_q and TFAP of
Eqs. TFAP, yTFAP, and the PCG iteration counts the paper reports for TFECS,
SECS and TFAP with the banded preconditioner (N_BW = 10)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import propagate as P
from oracle import stationary as ST
from oracle import tables as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold():
    return json.load(open(os.path.join(GOLD, "paper_test_setup.json")))


def test_tfap_profile_expansion():
    """Eq. yTFAP with a = c^3 - 16, b = c^3 - 17: expanding 4/(1-s)^2 -
    4/(1+s)^2 = 16 s + 32 s^3 + 48 s^5 + ... gives y(s) = c s + (49 - c^3)/c^2
    s^3 + O(s^5) (the linear onset the paper contrasts with ytilde ~ s^3),
    and a double pole y(s) (1 - s)^2 -> 4/c^2 at the box edge."""
    c = gold()["tfap_c"]
    for s in (1e-4, 1e-3):
        assert abs(T.tfap_y(s) / s - c) < 5 * s * s * abs((49 - c ** 3) / c ** 2) + 1e-9
    s = 2e-3
    cub = (T.tfap_y(s) - c * s) / s ** 3
    assert abs(cub - (49 - c ** 3) / c ** 2) < 1e-2
    for e in (1e-6, 1e-7):
        s = 1.0 - e
        assert abs(T.tfap_y(s) * e * e - 4.0 / c ** 2) < 1e-4


def test_absorbers_are_absorbing_and_unscaled():
    """Both absorbers leave the contour real (q = 1, z = x, so C = 0) and have
    Im U_a <= 0, vanishing inside r_s; the linear CAP's real part
    E_CAP (1 - cos 2 phi) is >= 0."""
    g = gold()
    n, rmax, rs = g["N"], g["rmax"], g["r_s"]
    x, _ = T.grid(n, -rmax, rmax)
    for kind in (T.CAP, T.TFAP):
        assert np.all(T.q_contour(x, kind, rs, rmax, math.pi / 4) == 1.0)
        assert np.all(T.z_contour(x, kind, rs, rmax, math.pi / 4) == x)
        Cs, Cd, Cu = T.c_tridiag(n, -rmax, rmax, kind, rs, math.pi / 4)
        assert max(np.abs(Cs).max(), np.abs(Cd).max(), np.abs(Cu).max()) == 0.0
        u = T.absorbing_potential(x, kind, rs, rmax, math.pi / 4, g["cap_energy"], g["tfap_kmin"])
        assert np.all(u.imag <= 0.0) and np.all(u[np.abs(x) <= rs] == 0.0)
        assert u.imag.min() < 0.0
    u = T.absorbing_potential(x, T.CAP, rs, rmax, math.pi / 4, 2.0)
    assert np.all(u.real >= 0.0)


def test_absorbers_dissipate_norm():
    """With Im U <= 0 every factor of the split step has modulus <= 1, so the
    norm never grows; it falls once the packet reaches the absorber.  With the
    absorber switched off (E_CAP = 0, k_min = 0) the step is unitary."""
    g = gold()
    n, rmax, rs, v0 = g["N"], g["rmax"], g["r_s"], g["v0"]
    for kind, kw, off in ((T.CAP, "e_cap", {"e_cap": 0.0}), (T.TFAP, "kmin", {"kmin": 0.0})):
        p = P.Problem1D(n, -rmax, rmax, rs, theta=math.pi / 4, kind=kind, dt=0.01, potential=False,
                        e_cap=g["cap_energy"], kmin=g["tfap_kmin"])
        psi = math.pi ** -0.25 * np.exp(-p.x ** 2 / 2 + 1j * v0 * p.x)
        norms = [p.h * np.sum(np.abs(psi) ** 2)]
        for _ in range(20):
            psi = p.step(psi, 100)
            norms.append(p.h * np.sum(np.abs(psi) ** 2))
        assert all(b <= a * (1 + 1e-13) for a, b in zip(norms, norms[1:]))
        assert norms[-1] < 0.8 * norms[0]
        q = P.Problem1D(n, -rmax, rmax, rs, theta=math.pi / 4, kind=kind, dt=0.01, potential=False, **off)
        psi = math.pi ** -0.25 * np.exp(-q.x ** 2 / 2 + 1j * v0 * q.x)
        n0 = q.h * np.sum(np.abs(psi) ** 2)
        psi = q.step(psi, 500)
        assert abs(q.h * np.sum(np.abs(psi) ** 2) - n0) < 1e-12


def _interior_error(kind, tt=20.0):
    g = gold()
    n, rmax, rs, v0 = g["N"], g["rmax"], g["r_s"], g["v0"]
    p = P.Problem1D(n, -rmax, rmax, rs, theta=math.pi / 4, kind=kind, alpha=g["tfecs_alpha"],
                    dt=0.0, potential=False, e_cap=g["cap_energy"], kmin=g["tfap_kmin"])
    p.dt = p.h * p.h
    psi0 = math.pi ** -0.25 * np.exp(-p.x ** 2 / 2 + 1j * v0 * p.x)
    psi = p.step(psi0, int(round(tt / p.dt)))
    s2 = 1.0 + 1j * tt                               # free Gaussian, sigma = 1
    ex = (math.pi ** -0.25 * s2 ** -0.5 * np.exp(-(p.x - v0 * tt) ** 2 / (2 * s2)
                                                 + 1j * v0 * p.x - 0.5j * v0 * v0 * tt))
    m = np.abs(p.x) < rs
    return math.sqrt(p.h) * np.linalg.norm((psi - ex)[m]), p, psi


@pytest.mark.slow
def test_absorber_accuracy_ordering():
    """Sec. IV: the linear CAP distorts the result most, TFAP less, "even the
    simple SECS" suppresses the unphysical reflection much better than TFAP,
    and TFECS does best.  In the unscaled region the exact outgoing solution
    is the free packet, so the L2 distance to it there measures what the
    absorber reflects by t_max = 20 (measured: 3.7e-3, 2.7e-3, 8e-5, 3e-9)."""
    e_cap, _, _ = _interior_error(T.CAP)
    e_tfap, _, _ = _interior_error(T.TFAP)
    e_secs, _, _ = _interior_error(T.SECS)
    e_tfecs, _, _ = _interior_error(T.TFECS)
    assert e_tfecs < e_secs < e_tfap < e_cap
    assert e_secs < 0.1 * e_tfap


@pytest.mark.slow
def test_pcg_iteration_counts_on_paper_test():
    """Sec. IV, closing remarks: with N = 1024 and the banded preconditioner
    (N_l = 10), PCG to a discrepancy of 1e-12 took about 79 iterations on
    average for TFECS, 36 for SECS and 20 for TFAP.  The right-hand side is
    the wave function at t_max = 20 (E-SURFF), the spectrum points
    E = k^2/2 for k = 0.2 .. 6.  SECS and TFECS must fall within a third of
    the paper's counts (measured 34 and 89).  For TFAP (Eq. yTFAP as
    printed, k_min = 0.25, whose banded preconditioner reduces to the plain
    one since q = 1) the paper gives neither k_min nor the spectrum points of
    its count: it must be within a factor 2 of it (measured 32) and below
    TFECS."""
    g = gold()
    c = g["claims"]
    ks = np.arange(1, 31) * 0.2
    means = {}
    for kind, key in ((T.TFAP, "pcg_iterations_tfap"), (T.SECS, "pcg_iterations_secs"),
                      (T.TFECS, "pcg_iterations_tfecs")):
        _, p, psi = _interior_error(kind)
        st = ST.Stationary1D(p, nbw=g["N_BW"])
        its = []
        for k in ks:
            E = 0.5 * k * k
            _, it, hist = ST.cocg(lambda v: st.apply_A(v, E), lambda r: st.precond_band(r, E), psi,
                                  tol=g["pcg_tolerance"], maxit=2000)
            assert hist[-1] < g["pcg_tolerance"]
            its.append(it)
        means[key] = float(np.mean(its))
        if kind == T.TFAP:
            assert c[key] / 2 < means[key] < 2 * c[key], (key, means[key])
        else:
            assert abs(means[key] - c[key]) < c[key] / 3.0, (key, means[key])
    assert means["pcg_iterations_secs"] < means["pcg_iterations_tfecs"]
    assert means["pcg_iterations_tfap"] < means["pcg_iterations_tfecs"]
