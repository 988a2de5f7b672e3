"""Pins of the amplitude-extraction oracle (t&E-SURFF, Sec. I and Sec. IV):
the time-integration rules against closed forms, and the amplitudes of the
paper's own test against the spectrum of Eq. Ateor at the accuracy levels
the paper reports (Sec. IV)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import propagate as P
from oracle import stationary as ST
from oracle import surff as SF
from oracle import tables as T

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_test_setup.json")))


def test_filon_is_exact_for_quadratics_times_the_exponential():
    """Filon-Simpson integrates e^{i w t} q(t) exactly for a quadratic q,
    whatever w tau (closed form by parts); Simpson does so only for w = 0."""
    a, b, c = 0.3 - 0.2j, -1.1 + 0.4j, 0.7 + 0.05j
    tau, M = 0.05, 40
    t = tau * np.arange(M + 1)
    q = a + b * t + c * t * t
    for w in (0.0, 0.3, 7.0, 60.0):
        if w == 0.0:
            ex = a * t[-1] + b * t[-1] ** 2 / 2 + c * t[-1] ** 3 / 3
        else:
            T_ = t[-1]
            e = np.exp(1j * w * T_)
            # int_0^T e^{iwt} t^p dt, p = 0, 1, 2, by parts
            i0 = (e - 1) / (1j * w)
            i1 = (T_ * e - i0) / (1j * w)
            i2 = (T_ * T_ * e - 2 * i1) / (1j * w)
            ex = a * i0 + b * i1 + c * i2
        assert abs(SF.time_integral(q, tau, w, rule="filon") - ex) < 1e-12 * max(1.0, abs(ex))
    assert abs(SF.time_integral(q, tau, 0.0, rule="simpson") - (a * t[-1] + b * t[-1] ** 2 / 2
                                                              + c * t[-1] ** 3 / 3)) < 1e-12


def test_simpson_is_fourth_order():
    """Simpson's rule on e^{i w t} e^{-t}: error falls 16x per halving of tau."""
    w, T_ = 3.0, 2.0
    ex = (np.exp((1j * w - 1) * T_) - 1) / (1j * w - 1)
    errs = []
    for M in (20, 40, 80):
        t = np.linspace(0, T_, M + 1)
        errs.append(abs(SF.time_integral(np.exp(-t), T_ / M, w, rule="simpson") - ex))
    assert 14 < errs[0] / errs[1] < 18 and 14 < errs[1] / errs[2] < 18


def _paper_case(n, kind, tmax):
    rmax, rs, v0 = GOLD["rmax"], GOLD["r_s"], GOLD["v0"]
    p = P.Problem1D(n, -rmax, rmax, rs, theta=math.pi / 4, kind=kind, alpha=GOLD["tfecs_alpha"],
                    dt=0.0, potential=False)
    p.dt = p.h * p.h                                     # tau = h^2 (Sec. IV)
    psi0 = math.pi ** -0.25 * np.exp(-p.x ** 2 / 2 + 1j * v0 * p.x)   # Eq. psi0
    nst = int(round(tmax / p.dt))
    nst += nst % 2
    samp, psiT = SF.record(p, psi0, nst)
    st = ST.Stationary1D(p, nbw=GOLD["N_BW"])
    w = SF.surface_weights(p.x, p.k, rs)

    def amp(kk, rule="filon"):
        E = 0.5 * kk * kk
        phi, _, hist = ST.cocg(lambda v: st.apply_A(v, E), lambda r: st.precond_band(r, E), psiT,
                               tol=1e-14, maxit=5000)
        ap, am = SF.amplitudes(samp, phi, E, rs, p.dt, rule=rule, weights=w)
        return ap if kk > 0 else am
    return amp, v0


@pytest.mark.slow
def test_tfecs_amplitudes_match_the_packet_spectrum():
    """Sec. IV: with TFECS the amplitude error is of order 1e-6.  Pure
    E-SURFF (t_max = 0) and t&E-SURFF at t_max = 20 (half the packet in the
    scaled region) both reproduce Eq. Ateor for 1 <= |k| <= 6 at N = 1024,
    and agree with each other (the two parts trade places, the sum is
    invariant)."""
    a0, v0 = _paper_case(1024, T.TFECS, 0.0)
    a20, _ = _paper_case(1024, T.TFECS, 20.0)
    for kk in (-6.0, -3.0, -1.0, 1.0, 2.0, 3.0, 4.5, 6.0):
        x0, x20 = a0(kk), a20(kk)
        assert abs(x0 - SF.a_teor(kk, v0)) < 2e-6, kk
        assert abs(x20 - SF.a_teor(kk, v0)) < 2e-6, kk
        assert abs(x20 - x0) < 5e-7, kk


@pytest.mark.slow
def test_secs_error_level_and_ordering():
    """Sec. IV: SECS leaves an amplitude error of ~1e-4 from unphysical
    reflection for k < -2.5, TFECS far less."""
    s20, v0 = _paper_case(1024, T.SECS, 20.0)
    t20, _ = _paper_case(1024, T.TFECS, 20.0)
    ks = (-6.0, -5.0, -4.0, -3.0)
    es = [abs(s20(k) - SF.a_teor(k, v0)) for k in ks]
    et = [abs(t20(k) - SF.a_teor(k, v0)) for k in ks]
    assert 3e-5 < max(es) < 3e-4
    assert max(et) < 1e-2 * max(es)


@pytest.mark.slow
def test_filon_beats_simpson_at_large_k():
    """Sec. IV, closing remarks: with tau = h^2 the Simpson error of the
    flux integral grows with |k| (the flux oscillates like e^{iEt}); the
    Filon-Simpson rule does not.  N = 512, t_max = 20, k = 6."""
    a, v0 = _paper_case(512, T.TFECS, 20.0)
    es = abs(a(6.0, "simpson") - SF.a_teor(6.0, v0))
    ef = abs(a(6.0, "filon") - SF.a_teor(6.0, v0))
    assert ef < es / 5
