"""Parity after a whole propagation, in the launch configurations the
benchmark times.

  - The laser batch: one sampled instance of each size (N = 2048 .. 16384)
    advanced over the whole pulse (22046 steps of dt = 0.02) by one batch plan,
    against the oracle's literal 4-FFT steps: complex128 to 1e-11.  The same
    instances in complex64 are compared with the same oracle runs: the FP32
    target 1e-5 is not met after the whole pulse (a slow, mostly norm-like
    drift of 1e-8 per step remains after every fixed table and constant was
    made exact to ~2^-48), so that case is an expected failure and a guard
    holds the measured level.
  - The 2D workload's contour and potential (box [-200, 200]^2, sharp
    theta = 0.4, U = -1/sqrt(x^2 + y^2 + 1), four seeded Gaussians) on a
    256^2 grid for its whole 10000 steps, and on the full 2048^2 grid for
    200 steps: complex128 to 1e-11.
  - The 3D workload's contour and potential ([-40, 40]^3, sharp theta = 0.4,
    U = -1/sqrt(r^2 + 1), four seeded Gaussians) on a 64^3 grid for 1000
    steps: complex128 to 1e-11.
The error is relative to the oracle's state at the end (its norm stays
above 0.5 here)."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

import paper_1505_06707_gb300 as S  # noqa: E402
import workloads as W  # noqa: E402
from oracle import propagate as P  # noqa: E402

CT = {S.SOFT_C64: torch.complex64, S.SOFT_C128: torch.complex128}
C64_GUARD = 5e-4          # measured 0.8 - 2.2e-4 after the whole pulse


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    S.load()


@pytest.fixture(scope="module")
def w2_case():
    ws = [next(w for w in (W.w2_instance(j) for j in range(256)) if w["n"] == n) for n in W.W2_SIZES]
    nst = W.w2_nsteps()
    probs = [P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], kind=w["contour"],
                         a2=w["a2"], dt=w["dt"]) for w in ws]
    refs = P.step_batch(probs, [w["psi0"] for w in ws], nst,
                        fields=[(w["E0"], w["omega"], w["ncyc"]) for w in ws])
    return ws, nst, refs


def w2_gpu(ws, nst, prec):
    plan = S.soft_create_batch([w["n"] for w in ws], [(w["a"], w["b"]) for w in ws],
                               [w["R0"] for w in ws], [w["theta"] for w in ws],
                               [(w["E0"], w["omega"], w["ncyc"]) for w in ws], W.W2_DT,
                               prec=prec, contour=W.W2_CONTOUR, autotune=1)
    try:
        offs, _ = S.soft_batch_layout(plan)
        d = torch.tensor(np.concatenate([w["psi0"] for w in ws]), dtype=CT[prec], device="cuda")
        t = S.soft_step_batch(plan, d, nst, 0.0)
        torch.cuda.synchronize()
        assert abs(t - nst * W.W2_DT) < 1e-9
        h = d.cpu().numpy().astype(np.complex128)
        return [h[o:o + w["n"]] for o, w in zip(offs, ws)]
    finally:
        S.soft_destroy(plan)


def test_w2_whole_pulse_c128(w2_case):
    ws, nst, refs = w2_case
    for w, g, r in zip(ws, w2_gpu(ws, nst, S.SOFT_C128), refs):
        assert np.linalg.norm(r) * np.sqrt(w["b"] - w["a"]) / np.sqrt(w["n"]) > 0.5
        assert relerr(g, r) < 1e-11, (w["n"], relerr(g, r))


def test_w2_whole_pulse_c64_guard(w2_case):
    ws, nst, refs = w2_case
    errs = [relerr(g, r) for g, r in zip(w2_gpu(ws, nst, S.SOFT_C64), refs)]
    print("complex64 rel-L2 after the whole pulse, N = 2048 .. 16384:", errs)
    assert max(errs) < C64_GUARD


@pytest.mark.xfail(reason="complex64 misses the 1e-5 target after 22046 steps (measured 0.8-2.2e-4)",
                   strict=False)
def test_w2_whole_pulse_c64_target(w2_case):
    ws, nst, refs = w2_case
    errs = [relerr(g, r) for g, r in zip(w2_gpu(ws, nst, S.SOFT_C64), refs)]
    assert max(errs) < 1e-5


def w3_gpu(w, nst):
    plan = S.soft_create((w["nx"], w["ny"]), w["box"], w["R0"], w["theta"], w["dt"], prec=S.SOFT_C128,
                         soft_a2=w["a2"])
    try:
        d = torch.tensor(w["psi0"], dtype=torch.complex128, device="cuda")
        S.soft_step(plan, d, nst, 0.0)
        torch.cuda.synchronize()
        return d.cpu().numpy()
    finally:
        S.soft_destroy(plan)


def test_w3_contour_whole_run_on_256sq():
    w = W.w3(n=256)
    ref = P.Problem2D(w["nx"], w["ny"], w["box"], w["R0"], theta=w["theta"], a2=w["a2"],
                      dt=w["dt"]).step(w["psi0"], w["nsteps"])
    got = w3_gpu(w, w["nsteps"])
    assert np.linalg.norm(ref) * (400.0 / 256) > 0.5
    assert relerr(got, ref) < 1e-11


def test_w3_full_size_200_steps_c128():
    w = W.w3()
    nst = 200
    ref = P.Problem2D(w["nx"], w["ny"], w["box"], w["R0"], theta=w["theta"], a2=w["a2"],
                      dt=w["dt"]).step(w["psi0"], nst)
    assert relerr(w3_gpu(w, nst), ref) < 1e-11


def test_w6_contour_1000_steps_on_64cube():
    w = W.w6(n=64)
    psi0 = W.w6_state(w["n"], w["box"], seed=0)
    nst = 1000
    ref = P.Problem3D(w["n"], w["box"], w["R0"], theta=w["theta"], kind=w["kind"], a2=w["a2"],
                      dt=w["dt"]).step(psi0, nst)
    plan = S.soft_create(w["n"], w["box"], w["R0"], w["theta"], w["dt"], prec=S.SOFT_C128,
                         contour=w["kind"], soft_a2=w["a2"])
    try:
        d = torch.tensor(psi0, dtype=torch.complex128, device="cuda")
        S.soft_step(plan, d, nst, 0.0)
        torch.cuda.synchronize()
        got = d.cpu().numpy()
    finally:
        S.soft_destroy(plan)
    h = 80.0 / 64
    assert np.linalg.norm(ref) * h ** 1.5 > 0.5
    assert relerr(got, ref) < 1e-11
