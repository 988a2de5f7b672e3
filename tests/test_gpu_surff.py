"""GPU parity of the amplitude extraction of the paper's test (t&E-SURFF,
Sec. I and Sec. IV): the surface samples that the step kernel takes from
its spectrum after every step, and the amplitudes from the flux integral
and the stationary solutions, against the oracle (oracle/surff.py) and
against the packet spectrum of Eq. Ateor."""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1505_06707_gb300 as S  # noqa: E402
from oracle import propagate as P  # noqa: E402
from oracle import stationary as ST  # noqa: E402
from oracle import surff as SF  # noqa: E402
from oracle import tables as T  # noqa: E402

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_test_setup.json")))
KIND = {T.SECS: S.CONTOUR_SECS, T.TFECS: S.CONTOUR_TFECS}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    S.load()


def paper(n, kind, potential=False):
    rmax, rs = G["rmax"], G["r_s"]
    h = 2 * rmax / n
    plan = S.soft_create(n, (-rmax, rmax), rs, math.pi / 4, h * h, prec=S.SOFT_C128, contour=KIND[kind],
                         charge=1.0 if potential else 0.0, tfecs_alpha=G["tfecs_alpha"])
    p = P.Problem1D(n, -rmax, rmax, rs, theta=math.pi / 4, kind=kind, alpha=G["tfecs_alpha"], dt=h * h,
                    potential=potential)
    psi0 = math.pi ** -0.25 * np.exp(-p.x ** 2 / 2 + 1j * G["v0"] * p.x)
    return plan, p, psi0


def gpu_samples(plan, psi0, nsteps, field=None, chunks=1):
    d = torch.tensor(psi0, dtype=torch.complex128, device="cuda")
    samp = torch.zeros((nsteps + 1, 4), dtype=torch.complex128, device="cuda")
    t, done = 0.0, 0
    per = nsteps // chunks
    for c in range(chunks):
        k = per if c < chunks - 1 else nsteps - done
        t = S.soft_step_surface(plan, d, k, t, samp[done:], field=field)
        done += k
    torch.cuda.synchronize()
    return d, samp


@pytest.mark.parametrize("kind", [T.TFECS, T.SECS])
def test_surface_samples_match_oracle(kind):
    """The paper's grid (N = 1024, tau = h^2) over t_max = 20 (2000 steps):
    every sample psi(+-R), psi'(+-R) and the final state match the oracle."""
    plan, p, psi0 = paper(1024, kind)
    try:
        d, samp = gpu_samples(plan, psi0, 2000)
        ref, refT = SF.record(p, psi0, 2000)
        got = samp.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
        assert np.linalg.norm(d.cpu().numpy() - refT) < 1e-11 * np.linalg.norm(refT)
    finally:
        S.soft_destroy(plan)


def test_surface_samples_across_calls_chunks_and_a_field():
    """Sampling continues across calls and across the step kernel's
    4096-step chunks, with a laser field and the soft-Coulomb potential;
    the state equals soft_step's."""
    n = 256
    plan, p, psi0 = paper(n, T.TFECS, potential=True)
    field = (0.05, 0.5, 3.0)
    try:
        d, samp = gpu_samples(plan, psi0, 5000, field=field, chunks=2)
        ref, refT = SF.record(p, psi0, 5000, field=field)
        got = samp.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
        d2 = torch.tensor(psi0, dtype=torch.complex128, device="cuda")
        S.soft_step(plan, d2, 2500, 0.0, field=field)
        S.soft_step(plan, d2, 2500, 2500 * p.dt, field=field)
        torch.cuda.synchronize()
        assert torch.equal(d, d2)
    finally:
        S.soft_destroy(plan)


def test_amplitudes_match_oracle_and_the_packet_spectrum():
    """The whole extraction on the GPU (sampled propagation to t_max = 20,
    30 stationary solves with right-hand side psi(t_max), amplitudes by
    Simpson and Filon-Simpson) against the oracle's, and TFECS against
    Eq. Ateor within the paper's ~1e-6 for 1 <= |k| <= 6."""
    n = 1024
    plan, p, psi0 = paper(n, T.TFECS)
    try:
        d, samp = gpu_samples(plan, psi0, 2000)
        ks = np.arange(1, 31) * 0.2
        Es = [0.5 * k * k for k in ks]
        phi = torch.zeros((len(Es), n), dtype=torch.complex128, device="cuda")
        rc, its, rr = S.sse_pcg_solve(plan, Es, d, phi, tol=1e-13, maxit=3000, precond=1)
        assert rc == 0
        ref_s, refT = SF.record(p, psi0, 2000)
        st = ST.Stationary1D(p, nbw=10)
        w = SF.surface_weights(p.x, p.k, p.R0)
        for rule_i, rule in ((0, "simpson"), (1, "filon")):
            amp = S.sse_surff(plan, Es, phi, samp, t0=0.0, rule=rule_i).cpu().numpy()
            for e in (0, 4, 9, 14, 19, 29):
                E = Es[e]
                phi_o, _, _ = ST.cocg(lambda v: st.apply_A(v, E), lambda r: st.precond_band(r, E), refT,
                                      tol=1e-13, maxit=3000)
                ap, am = SF.amplitudes(ref_s, phi_o, E, p.R0, p.dt, rule=rule, weights=w)
                assert abs(amp[e, 0] - ap) < 1e-9 and abs(amp[e, 1] - am) < 1e-9, (rule, e)
            k = ks
            sel = k >= 1.0 - 1e-9
            errp = np.abs(amp[sel, 0] - SF.a_teor(k[sel], G["v0"]))
            errm = np.abs(amp[sel, 1] - SF.a_teor(-k[sel], G["v0"]))
            assert errp.max() < 2e-6 and errm.max() < 2e-6, (rule, errp.max(), errm.max())
    finally:
        S.soft_destroy(plan)
