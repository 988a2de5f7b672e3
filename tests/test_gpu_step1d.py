"""GPU parity of the 1D ECS split-operator step (Sec. II) against the oracle,
through the C ABI.

Bars.  complex128: rel-L2 <= 1e-11 after the full propagation.  complex64:
1e-5, the FP32 target, for every run here (up to the 2000 steps of the 1D
workload, measured 5e-6 there).  The FP32 FFT applies its constant
rotations and pass twiddles as compensated hi+lo products: a rounded
(cos, sin) pair has |w| != 1 and, applied at the same positions in every
step, gave a coherent drift of ~1e-7 per step before.  The whole 22046-step
pulse of the laser workload is covered by test_gpu_full_propagation."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1505_06707_gb300 as S  # noqa: E402
import workloads as W  # noqa: E402
from oracle import observe as O  # noqa: E402
from oracle import propagate as P  # noqa: E402
from oracle import tables as T  # noqa: E402

CT = {S.SOFT_C64: torch.complex64, S.SOFT_C128: torch.complex128}


def tol(prec, nsteps=None, n=None):
    return 1e-11 if prec == S.SOFT_C128 else 1e-5


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_run(n, box, R0, theta, dt, psi0, nsteps, prec=S.SOFT_C128, field=None, t0=0.0,
            chunks=1, **opt):
    plan = S.soft_create(n, box, R0, theta, dt, prec=prec, **opt)
    try:
        d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
        t = t0
        per = nsteps // chunks
        for c in range(chunks):
            k = per if c < chunks - 1 else nsteps - per * (chunks - 1)
            t = S.soft_step(plan, d, k, t, field=field)
        torch.cuda.synchronize()
        assert abs(t - (t0 + nsteps * dt)) < 1e-9 * max(1.0, abs(t))
        return d.cpu().numpy().astype(np.complex128)
    finally:
        S.soft_destroy(plan)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    S.load()


def test_w1_full_run_c128():
    """The 1D workload (N=1024, sharp ECS theta=0.5, soft-Coulomb, 2000 steps)
    matches the oracle to 1e-11."""
    w = W.w1()
    ref = P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], a2=w["a2"],
                      dt=w["dt"]).step(w["psi0"], w["nsteps"])
    got = gpu_run(w["n"], (w["a"], w["b"]), w["R0"], w["theta"], w["dt"], w["psi0"], w["nsteps"])
    assert relerr(got, ref) < 1e-11


def test_w1_full_run_c64():
    w = W.w1()
    ref = P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], a2=w["a2"],
                      dt=w["dt"]).step(w["psi0"], w["nsteps"])
    got = gpu_run(w["n"], (w["a"], w["b"]), w["R0"], w["theta"], w["dt"], w["psi0"], w["nsteps"],
                  prec=S.SOFT_C64)
    err = relerr(got, ref)
    print("complex64 W1 rel-L2 after %d steps: %.3e" % (w["nsteps"], err))
    assert err < tol(S.SOFT_C64, w["nsteps"], w["n"])


def test_free_gaussian_closed_form_c128():
    """theta = 0, U = 0: the GPU must reproduce free spreading (closed form
    summed over periodic images), independent of the oracle."""
    n, a, b = 1024, -200.0, 200.0
    x = a + (b - a) / n * (np.arange(n) + 0.5)
    L = b - a

    def free(t):
        s2 = 25.0
        out = 0
        for m in range(-3, 4):
            xx = x + m * L
            out = out + ((s2 / math.pi) ** 0.25 * (s2 + 1j * t) ** -0.5
                         * np.exp(-(xx - t) ** 2 / (2 * (s2 + 1j * t)) + 1j * xx - 0.5j * t))
        return out
    got = gpu_run(n, (a, b), 150.0, 0.0, 0.05, free(0.0), 2000, charge=0.0)
    assert relerr(got, free(100.0)) < 1e-11


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384])
def test_random_state_all_sizes(n, prec):
    """Every built size and both precisions, random complex state, sharp ECS
    (strip = 1/8 of the box per side plus the coupled neighbours), 7 steps."""
    rng = np.random.default_rng(n + prec)
    psi0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    hw = 8.0 * n / 1024
    R0 = 0.75 * hw
    ref = P.Problem1D(n, -hw, hw, R0, theta=0.5, a2=2.0, dt=0.02).step(psi0, 7)
    got = gpu_run(n, (-hw, hw), R0, 0.5, 0.02, psi0, 7, prec=prec)
    assert relerr(got, ref) < (1e-12 if prec == S.SOFT_C128 else 2e-6)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("contour", [S.CONTOUR_SECS, S.CONTOUR_TFECS])
def test_smooth_contours(contour, prec):
    """SECS and TFECS contours (Eqs. qSECS, qTFECS) on the paper's own test
    grid (b = -a = 51.2, r_s = 40, N = 1024, tau = h^2)."""
    n, b, rs = 1024, 51.2, 40.0
    h = 2 * b / n
    x = -b + h * (np.arange(n) + 0.5)
    psi0 = math.pi ** -0.25 * np.exp(-x ** 2 / 2 + 2j * x)
    kind = T.SECS if contour == S.CONTOUR_SECS else T.TFECS
    nst = 500
    th = math.pi / 4                     # the paper's SECS final angle
    ref = P.Problem1D(n, -b, b, rs, theta=th, kind=kind, alpha=0.5, dt=h * h,
                      potential=False).step(psi0, nst)
    got = gpu_run(n, (-b, b), rs, th, h * h, psi0, nst, prec=prec, contour=contour, charge=0.0)
    assert relerr(got, ref) < tol(prec, nst, n)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("kind", [S.ABSORB_CAP, S.ABSORB_TFAP])
def test_comparison_absorbers(kind, prec):
    """The linear CAP (Eq. CAP_via_q, E_CAP = 2) and TFAP (Eqs. TFAP, yTFAP,
    k_min = 0.25) on the paper's test grid (b = -a = 51.2, r_s = 40,
    N = 1024, tau = h^2): real contour, complex potential, no strip."""
    n, b, rs = 1024, 51.2, 40.0
    h = 2 * b / n
    x = -b + h * (np.arange(n) + 0.5)
    psi0 = math.pi ** -0.25 * np.exp(-x ** 2 / 2 + 2j * x)
    okind = T.CAP if kind == S.ABSORB_CAP else T.TFAP
    nst = 2000                  # t_max = 20: half the packet is inside the absorber
    ref = P.Problem1D(n, -b, b, rs, theta=math.pi / 4, kind=okind, dt=h * h, potential=False,
                      e_cap=2.0, kmin=0.25).step(psi0, nst)
    assert np.linalg.norm(ref) < 0.95 * np.linalg.norm(psi0)        # the absorber has acted
    got = gpu_run(n, (-b, b), rs, math.pi / 4, h * h, psi0, nst, prec=prec, contour=kind, charge=0.0,
                  cap_energy=2.0, tfap_kmin=0.25)
    assert relerr(got, ref) < tol(prec, nst, n)
    plan = S.soft_create(n, (-b, b), rs, 0.5, h * h, prec=prec, contour=kind)
    try:
        d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
        with pytest.raises(S.SoftError):                                # absorbers take no field
            S.soft_step(plan, d, 1, 0.0, field=(0.05, 0.057, 4.0))
    finally:
        S.soft_destroy(plan)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_laser_field_single(prec):
    """One laser-batch instance (N = 2048, h = 1/64, SECS contour reaching
    theta = 0.5, pulse E0 sin^2 sin) for 300 steps from mid-pulse, split over
    three calls."""
    w = W.w2_instance(3)
    n = 2048
    hw = 8.0 * n / 1024
    x = -hw + 2 * hw / n * (np.arange(n) + 0.5)
    psi0 = np.exp(-x ** 2 / 3.0) * np.exp(0.3j * x)
    field = (0.08, W.W2_OMEGA, W.W2_NCYC)
    t0 = 100.0
    ref = P.Problem1D(n, -hw, hw, 0.75 * hw, theta=0.5, kind=T.SECS, a2=2.0,
                      dt=0.02).step(psi0, 300, t0=t0, field=field)
    got = gpu_run(n, (-hw, hw), 0.75 * hw, 0.5, 0.02, psi0, 300, prec=prec, field=field, t0=t0,
                  chunks=3, contour=S.CONTOUR_SECS)
    assert relerr(got, ref) < tol(prec, 300, n)
    del w


def test_nsteps_zero_is_noop_and_theta0_has_no_strip():
    n = 256
    rng = np.random.default_rng(0)
    psi0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = gpu_run(n, (-20.0, 20.0), 15.0, 0.5, 0.01, psi0, 0)
    assert np.array_equal(got, psi0)
    ref = P.Problem1D(n, -20.0, 20.0, 15.0, theta=0.0, dt=0.01).step(psi0, 5)
    got = gpu_run(n, (-20.0, 20.0), 15.0, 0.0, 0.01, psi0, 5)
    assert relerr(got, ref) < 1e-12


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_set_potential(prec):
    """soft_set_potential: a user potential (a complex-scaled Gaussian well
    plus a weak harmonic term, evaluated at z(x_i)) replaces the soft-Coulomb
    one; the oracle steps with the same U.  Also with a laser field, and
    setting the default back restores the default run."""
    n, hw, R0, th, dt, nst = 1024, 40.0, 30.0, 0.5, 0.02, 150
    ref = P.Problem1D(n, -hw, hw, R0, theta=th, a2=2.0, dt=dt)
    U_default = ref.U0.copy()
    U = -1.5 * np.exp(-ref.z ** 2 / 4.0) + 0.002 * ref.z ** 2
    x = ref.x
    psi0 = np.exp(-(x - 3.0) ** 2 / 4.0 + 0.8j * x)
    field = (0.04, 0.3, 2.0)
    plan = S.soft_create(n, (-hw, hw), R0, th, dt, prec=prec, soft_a2=2.0)
    try:
        S.soft_set_potential(plan, U)
        ref.U0 = U.copy()
        for fld in (None, field):
            d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
            S.soft_step(plan, d, nst, 0.0, field=fld)
            torch.cuda.synchronize()
            want = ref.step(psi0, nst, 0.0, field=fld)
            assert relerr(d.cpu().numpy().astype(np.complex128), want) < tol(prec, nst, n)
        S.soft_set_potential(plan, U_default)
        d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
        S.soft_step(plan, d, nst, 0.0)
        torch.cuda.synchronize()
        ref.U0 = U_default
        assert relerr(d.cpu().numpy().astype(np.complex128), ref.step(psi0, nst)) < tol(prec, nst, n)
        with pytest.raises(S.SoftError):
            S.soft_set_potential(plan, U[: n // 2])
        bad = U.copy()
        bad[7] = np.nan
        with pytest.raises(S.SoftError):
            S.soft_set_potential(plan, bad)
    finally:
        S.soft_destroy(plan)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_batch_mixed_sizes_with_fields(prec):
    """A batch of instances of the laser workload (mixed N, own E0 each)
    advanced in one call; each compared with its own oracle run."""
    idx = [0, 1, 2, 3, 5, 8, 13, 21]
    ws = [W.w2_instance(j) for j in idx]
    nst, t0 = 40, 50.0
    plan = S.soft_create_batch([w["n"] for w in ws], [(w["a"], w["b"]) for w in ws],
                               [w["R0"] for w in ws], [w["theta"] for w in ws],
                               [(w["E0"], w["omega"], w["ncyc"]) for w in ws], W.W2_DT, prec=prec,
                               contour=W.W2_CONTOUR)
    try:
        offs, tot = S.soft_batch_layout(plan)
        packed = np.concatenate([w["psi0"] for w in ws])
        assert tot == len(packed)
        d = torch.tensor(packed, dtype=CT[prec], device="cuda")
        S.soft_step_batch(plan, d, nst, t0)
        torch.cuda.synchronize()
        got = d.cpu().numpy().astype(np.complex128)
    finally:
        S.soft_destroy(plan)
    probs = [P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], kind=w["contour"],
                         a2=w["a2"], dt=w["dt"]) for w in ws]
    refs = P.step_batch(probs, [w["psi0"] for w in ws], nst, t0s=[t0] * len(ws),
                        fields=[(w["E0"], w["omega"], w["ncyc"]) for w in ws])
    for o, w, r in zip(offs, ws, refs):
        assert relerr(got[o:o + w["n"]], r) < tol(prec, nst, w["n"])


def test_observables_match_oracle():
    ws = [w for w in (W.w2_instance(j) for j in range(12)) if w["n"] <= 8192][:3]
    plan = S.soft_create_batch([w["n"] for w in ws], [(w["a"], w["b"]) for w in ws],
                               [w["R0"] for w in ws], [w["theta"] for w in ws], None, 0.02,
                               contour=W.W2_CONTOUR)
    try:
        rng = np.random.default_rng(4)
        states = [rng.standard_normal(w["n"]) + 1j * rng.standard_normal(w["n"]) for w in ws]
        d = torch.tensor(np.concatenate(states), dtype=torch.complex128, device="cuda")
        nrm = torch.zeros(3, dtype=torch.float64, device="cuda")
        flx = torch.zeros(6, dtype=torch.float64, device="cuda")
        S.soft_observe(plan, d, nrm, flx)
        torch.cuda.synchronize()
        nrm, flx = nrm.cpu().numpy(), flx.cpu().numpy()
    finally:
        S.soft_destroy(plan)
    for i, (w, st) in enumerate(zip(ws, states)):
        x, h = T.grid(w["n"], w["a"], w["b"])
        assert abs(nrm[i] - O.norm_inside(st, x, h, w["R0"])) < 1e-12 * nrm[i]
        fl = O.flux_at_edges(st, x, h, w["R0"])
        assert np.allclose(flx[2 * i:2 * i + 2], fl, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_autotuned_batch_matches_default(prec):
    """A batch plan whose kernel variants were chosen by timing (autotune)
    computes the same states as the default variants, and repeated calls
    (replayed from the captured graph) continue the propagation correctly."""
    idx = list(range(12))
    ws = [W.w2_instance(j) for j in idx]
    args = ([w["n"] for w in ws], [(w["a"], w["b"]) for w in ws], [w["R0"] for w in ws],
            [w["theta"] for w in ws], [(w["E0"], w["omega"], w["ncyc"]) for w in ws], W.W2_DT)
    packed = np.concatenate([w["psi0"] for w in ws])
    outs = []
    for tune in (0, 1):
        plan = S.soft_create_batch(*args, prec=prec, contour=W.W2_CONTOUR, autotune=tune)
        try:
            d = torch.tensor(packed, dtype=CT[prec], device="cuda")
            t = 20.0
            for _ in range(3):
                t = S.soft_step_batch(plan, d, 10, t)
            torch.cuda.synchronize()
            assert abs(t - 20.6) < 1e-12
            outs.append(d.cpu().numpy().astype(np.complex128))
        finally:
            S.soft_destroy(plan)
    probs = [P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], kind=w["contour"],
                         a2=w["a2"], dt=w["dt"]) for w in ws]
    refs = P.step_batch(probs, [w["psi0"] for w in ws], 30, t0s=[20.0] * len(ws),
                        fields=[(w["E0"], w["omega"], w["ncyc"]) for w in ws])
    offs = np.concatenate([[0], np.cumsum([w["n"] for w in ws])[:-1]])
    for out in outs:
        for o, w, r in zip(offs, ws, refs):
            assert relerr(out[o:o + w["n"]], r) < tol(prec, 30, w["n"])


@pytest.mark.parametrize("prec", [S.SOFT_C64, S.SOFT_C128])
def test_w2_full_batch_sampled(prec):
    """The whole laser batch (4096 instances, N = 2048 .. 16384) in one mixed
    batch plan advanced by one call of 256 steps, as the benchmark launches
    it (autotuned: persistent kernel or per-size kernels, whichever is
    faster); 8 sampled instances, two per size, compared with their own
    oracle runs."""
    ws = [W.w2_instance(j) for j in range(4096)]
    nst, t0 = 256, 0.0
    sample = []
    for n in W.W2_SIZES:
        sample += [i for i, w in enumerate(ws) if w["n"] == n][:2]
    plan = S.soft_create_batch([w["n"] for w in ws], [(w["a"], w["b"]) for w in ws],
                               [w["R0"] for w in ws], [w["theta"] for w in ws],
                               [(w["E0"], w["omega"], w["ncyc"]) for w in ws], W.W2_DT,
                               prec=prec, contour=W.W2_CONTOUR, autotune=1)
    try:
        offs, tot = S.soft_batch_layout(plan)
        d = torch.tensor(np.concatenate([w["psi0"] for w in ws]), dtype=CT[prec], device="cuda")
        S.soft_step_batch(plan, d, nst, t0)
        torch.cuda.synchronize()
        got = {i: d[offs[i]:offs[i] + ws[i]["n"]].cpu().numpy().astype(np.complex128) for i in sample}
    finally:
        S.soft_destroy(plan)
    sw = [ws[i] for i in sample]
    probs = [P.Problem1D(w["n"], w["a"], w["b"], w["R0"], theta=w["theta"], kind=w["contour"],
                         a2=w["a2"], dt=w["dt"]) for w in sw]
    refs = P.step_batch(probs, [w["psi0"] for w in sw], nst, t0s=[t0] * len(sw),
                        fields=[(w["E0"], w["omega"], w["ncyc"]) for w in sw])
    for i, w, r in zip(sample, sw, refs):
        assert relerr(got[i], r) < tol(prec, nst, w["n"]), (i, w["n"])


def test_nonfinite_state_reported_by_status_query():
    """A NaN in the input state reaches the instance's first element through
    the FFT; soft_step_status reports it once (then the flag is clear), and a
    finite run reports nothing."""
    n, a, b, R0 = 1024, -50.0, 50.0, 40.0
    x = a + (b - a) / n * (np.arange(n) + 0.5)
    psi0 = np.exp(-x ** 2 / 8.0 + 0.5j * x)
    for prec in (S.SOFT_C128, S.SOFT_C64):
        plan = S.soft_create(n, (a, b), R0, 0.5, 0.05, prec=prec)
        try:
            d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
            S.soft_step(plan, d, 5, 0.0)
            S.soft_step_status(plan)                 # finite: no error
            bad = psi0.copy()
            bad[700] = np.nan
            d = torch.tensor(bad, dtype=CT[prec], device="cuda")
            S.soft_step(plan, d, 3, 0.0)
            with pytest.raises(S.SoftError) as e:
                S.soft_step_status(plan)
            assert e.value.status == -8
            S.soft_step_status(plan)                 # cleared by the query
        finally:
            S.soft_destroy(plan)


def test_field_change_between_calls_on_a_side_stream():
    """Two calls on a non-blocking stream, queued back to back with different
    fields and no synchronisation between them: each call must run with its
    own field (the descriptor update is ordered on the stream)."""
    w = W.w2_instance(3)
    n = w["n"]
    f1 = (w["E0"], w["omega"], w["ncyc"])
    f2 = (0.5 * w["E0"], 1.5 * w["omega"], 2.0)
    prob = P.Problem1D(n, w["a"], w["b"], w["R0"], theta=w["theta"], kind=w["contour"],
                       a2=w["a2"], dt=w["dt"])
    ref = prob.step(w["psi0"], 200, t0=5.0, field=f1)
    ref = prob.step(ref, 40, t0=5.0 + 200 * w["dt"], field=f2)
    plan = S.soft_create(n, (w["a"], w["b"]), w["R0"], w["theta"], w["dt"], prec=S.SOFT_C128,
                         contour=w["contour"], soft_a2=w["a2"])
    try:
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            d = torch.tensor(w["psi0"], dtype=torch.complex128, device="cuda")
        t = S.soft_step(plan, d, 200, 5.0, field=f1, stream=st)
        t = S.soft_step(plan, d, 40, t, field=f2, stream=st)
        st.synchronize()
        got = d.cpu().numpy()
    finally:
        S.soft_destroy(plan)
    assert relerr(got, ref) < 1e-11


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_secs_zero_angle_reduces_to_the_unscaled_step(prec):
    """The SECS contour at theta = 0 is q = 1 (no strip): the GPU step must
    match the oracle's unscaled step (the plan tables take the theta -> 0
    limit of the SECS z(x))."""
    n, a, b, R0 = 1024, -50.0, 50.0, 40.0
    x = a + (b - a) / n * (np.arange(n) + 0.5)
    psi0 = np.exp(-(x + 5.0) ** 2 / 6.0 + 0.9j * x)
    ref = P.Problem1D(n, a, b, R0, theta=0.0, kind=T.SHARP, a2=2.0, dt=0.02).step(psi0, 100)
    got = gpu_run(n, (a, b), R0, 0.0, 0.02, psi0, 100, prec=prec, contour=S.CONTOUR_SECS)
    assert relerr(got, ref) < (1e-12 if prec == S.SOFT_C128 else 2e-6)


@pytest.mark.parametrize("prec", [S.SOFT_C64, S.SOFT_C128])
def test_persistent_batch_matches_group_kernels(prec):
    """A batch plan runs its instances of N = 2048 .. 16384 through the
    persistent kernel (packs of same-size instances from a queue, several
    instances per CTA on named barriers) and the rest through one kernel per
    size group, beside it.  Both must give exactly what one kernel per size
    group gives (the same arithmetic per instance), including part-filled
    packs and sizes outside the persistent kernel, and match the oracle."""
    ws = [W.w2_instance(j) for j in range(37)]
    extra = []
    for n in (512, 1024):                   # sizes outside the persistent kernel
        hw = 8.0 * n / 1024
        x = -hw + 2 * hw / n * (np.arange(n) + 0.5)
        extra.append(dict(n=n, a=-hw, b=hw, R0=0.75 * hw, theta=0.5, contour=W.W2_CONTOUR, a2=2.0,
                          dt=W.W2_DT, E0=0.05, omega=W.W2_OMEGA, ncyc=W.W2_NCYC,
                          psi0=np.exp(-x ** 2 / 3.0 + 0.3j)))
    ws = ws[:20] + extra + ws[20:]
    args = ([w["n"] for w in ws], [(w["a"], w["b"]) for w in ws], [w["R0"] for w in ws],
            [w["theta"] for w in ws], [(w["E0"], w["omega"], w["ncyc"]) for w in ws], W.W2_DT)
    packed = np.concatenate([w["psi0"] for w in ws])
    outs = []
    for pers in (1, 0):
        plan = S.soft_create_batch(*args, prec=prec, contour=W.W2_CONTOUR, persistent=pers)
        try:
            d = torch.tensor(packed, dtype=CT[prec], device="cuda")
            t = 3.0
            for _ in range(2):
                t = S.soft_step_batch(plan, d, 12, t)
            torch.cuda.synchronize()
            outs.append(d.cpu().numpy())
            if pers:
                assert S.soft_last_launches(plan) == 5   # table, persistent, 2 groups, time
        finally:
            S.soft_destroy(plan)
    assert np.array_equal(outs[0], outs[1])
    sample = [0, 5, 20, 21, 30, len(ws) - 1]
    probs = [P.Problem1D(ws[i]["n"], ws[i]["a"], ws[i]["b"], ws[i]["R0"], theta=ws[i]["theta"],
                         kind=ws[i]["contour"], a2=ws[i]["a2"], dt=ws[i]["dt"]) for i in sample]
    refs = P.step_batch(probs, [ws[i]["psi0"] for i in sample], 24, t0s=[3.0] * len(sample),
                        fields=[(ws[i]["E0"], ws[i]["omega"], ws[i]["ncyc"]) for i in sample])
    offs = np.concatenate([[0], np.cumsum([w["n"] for w in ws])[:-1]])
    for i, r in zip(sample, refs):
        assert relerr(outs[0][offs[i]:offs[i] + ws[i]["n"]].astype(np.complex128), r) < tol(prec)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("n,nsteps", [(1024, 1), (1024, 2), (1024, 3), (16384, 1), (16384, 2)])
def test_call_lengths_1d(n, nsteps, prec):
    """Calls of 1 step (the first step is also the last: both half kinetic
    factors in one step), 2 steps (no middle step) and 3 steps, in a laser
    field, on the shared-memory and the N = 16384 configurations."""
    rng = np.random.default_rng(n + 31 * nsteps)
    psi0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    hw = 8.0 * n / 1024
    R0 = 0.75 * hw
    field, t0 = (0.05, 0.057, 4.0), 100.0
    ref = P.Problem1D(n, -hw, hw, R0, theta=0.5, kind=T.SECS, a2=2.0, dt=0.02).step(
        psi0, nsteps, t0=t0, field=field)
    got = gpu_run(n, (-hw, hw), R0, 0.5, 0.02, psi0, nsteps, prec=prec, field=field, t0=t0,
                  contour=S.CONTOUR_SECS)
    assert relerr(got, ref) < (1e-12 if prec == S.SOFT_C128 else 2e-6)
