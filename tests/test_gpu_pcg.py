"""GPU parity of the stationary solver (Sec. III): the A application
(Eq. linsys), the simple FFT preconditioner (Eq. PreconFFT) and the banded
ECS preconditioner (Eq. PreconFFT_ECS) against the oracle, and complex-
symmetric CG solves whose residual is recomputed by the oracle's own A."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1505_06707_gb300 as S  # noqa: E402
import workloads as W  # noqa: E402
from oracle import propagate as P  # noqa: E402
from oracle import stationary as ST  # noqa: E402
from oracle import tables as T  # noqa: E402


# the solver stops on the true FP64 residual f - A x (< 1e-8); recomputed
# with the oracle's A (numpy FFTs, another rounding order) it may differ
# from the solver's own evaluation by rounding only
TRUE_RES_TOL = 1e-8 * (1 + 1e-4)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    S.load()


def setup(n=256, box=(-40.0, 40.0, -40.0, 40.0), R0=30.0, theta=0.4, a2=1.0, charge=1.0):
    plan = S.soft_create((n, n), box, R0, theta, 0.02, prec=S.SOFT_C128, soft_a2=a2, charge=charge)
    p2 = P.Problem2D(n, n, box, R0, theta=theta, a2=a2, charge=charge, dt=0.02,
                     potential=charge != 0.0)
    st = ST.Stationary2D(p2, nbw=10, kind=T.SHARP, R0=R0, theta=theta)
    return plan, p2, st


def dev(a):
    return torch.tensor(a, dtype=torch.complex128, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_apply_A_and_preconditioners_match_oracle():
    plan, p2, st = setup()
    try:
        rng = np.random.default_rng(11)
        x = rng.standard_normal((256, 256)) + 1j * rng.standard_normal((256, 256))
        dx, dy = dev(x), dev(np.zeros_like(x))
        for E in (0.3, 1.7):
            S.sse_apply_A(plan, E, dx, dy)
            assert relerr(host(dy), st.apply_A(x, E)) < 1e-12
            # A computing in FP32 on complex64: 2^-24 per operation over the
            # two FFT pairs (compared with A of the rounded input)
            x32 = x.astype(np.complex64)
            y32 = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
            S.sse_apply_A32(plan, E, torch.from_numpy(x32).cuda(), y32)
            assert relerr(host(y32).astype(np.complex128), st.apply_A(x32.astype(np.complex128), E)) < 5e-6
            S.sse_apply_precond(plan, E, 0, dx, dy)
            assert relerr(host(dy), st.precond_simple(x, E)) < 1e-11
            S.sse_apply_precond(plan, E, 1, dx, dy)
            assert relerr(host(dy), st.precond_band(x, E)) < 1e-11
            # the same operator computing in FP32: rounding of 2^-24 per operation
            # over the ~20 FFT stages and band products of the three passes
            S.sse_apply_precond(plan, E, 4, dx, dy)
            assert relerr(host(dy), st.precond_band(x, E)) < 2e-5
    finally:
        S.soft_destroy(plan)


def test_set_potential_reaches_the_solver():
    """soft_set_potential after the solver's tables exist: A (FP64 and FP32)
    must use the new U (oracle A with the same U)."""
    plan, p2, st = setup()
    try:
        rng = np.random.default_rng(12)
        x = rng.standard_normal((256, 256)) + 1j * rng.standard_normal((256, 256))
        dx, dy = dev(x), dev(np.zeros_like(x))
        S.sse_apply_A(plan, 0.6, dx, dy)                      # builds the tables
        zx = T.z_contour(p2.x, T.SHARP, 30.0, 40.0, 0.4, 0.5)
        U = -2.0 * np.exp(-(zx[None, :] ** 2 + zx[:, None] ** 2) / 9.0) + 0.1j * np.cos(zx[:, None])
        S.soft_set_potential(plan, U)
        p2.U = np.ascontiguousarray(U, dtype=np.complex128)
        S.sse_apply_A(plan, 0.6, dx, dy)
        assert relerr(host(dy), st.apply_A(x, 0.6)) < 1e-12
        x32 = x.astype(np.complex64)
        y32 = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
        S.sse_apply_A32(plan, 0.6, torch.from_numpy(x32).cuda(), y32)
        assert relerr(host(y32).astype(np.complex128), st.apply_A(x32.astype(np.complex128), 0.6)) < 5e-6
    finally:
        S.soft_destroy(plan)


def test_pcg_fp32_preconditioner():
    """COCG (flexible beta) with the banded preconditioner computing in FP32
    (A, the residual and the dots stay FP64): every energy reaches the
    tolerance, checked with the oracle's A, in about the iterations of the
    FP64 preconditioner."""
    plan, p2, st = setup()
    try:
        n = 256
        xg = -40.0 + 80.0 / n * (np.arange(n) + 0.5)
        f = -np.exp(-(xg[None, :] ** 2 + (xg[:, None] - 3.0) ** 2) / 32.0).astype(np.complex128)
        Es = [0.2, 0.55, 1.1, 1.9]
        out = torch.zeros((len(Es), n, n), dtype=torch.complex128, device="cuda")
        rc1, its1, _ = S.sse_pcg_solve(plan, Es, dev(f), out, tol=1e-8, maxit=2000, precond=1)
        rc4, its4, rr4 = S.sse_pcg_solve(plan, Es, dev(f), out, tol=1e-8, maxit=2000, precond=4)
        assert rc1 == 0 and rc4 == 0, (rc4, its4, rr4)
        xs = host(out)
        for e, E in enumerate(Es):
            res = np.linalg.norm(st.apply_A(xs[e], E) - f) / np.linalg.norm(f)
            assert res < TRUE_RES_TOL, (E, res, its4[e])
            # FP32 rounding leaves the preconditioner inexact and not exactly
            # symmetric; measured cost up to ~25 % more iterations
            assert its4[e] <= 1.3 * its1[e] + 5, (its1, its4)
        print("iterations FP64 band", its1, "FP32 band", its4)
    finally:
        S.soft_destroy(plan)


def test_pcg_mixed_precision_reliable_updates():
    """precond 5: A and the banded preconditioner computing in FP32 on
    complex64 vectors, the residual replaced by the true FP64 one each time
    it has dropped tenfold.  Every energy must reach the tolerance on the
    oracle's A (so the reported residual is the true one), in about the
    iterations of the FP64 solve."""
    plan, p2, st = setup()
    try:
        n = 256
        xg = -40.0 + 80.0 / n * (np.arange(n) + 0.5)
        f = -np.exp(-(xg[None, :] ** 2 + (xg[:, None] - 3.0) ** 2) / 32.0).astype(np.complex128)
        Es = [0.2, 0.55, 1.1, 1.9]
        out = torch.zeros((len(Es), n, n), dtype=torch.complex128, device="cuda")
        rc1, its1, _ = S.sse_pcg_solve(plan, Es, dev(f), out, tol=1e-8, maxit=2000, precond=1)
        for tol in (1e-8, 1e-10):
            rc5, its5, rr5 = S.sse_pcg_solve(plan, Es, dev(f), out, tol=tol, maxit=2000, precond=5)
            assert rc5 == 0, (tol, rc5, its5, rr5)
            xs = host(out)
            for e, E in enumerate(Es):
                res = np.linalg.norm(st.apply_A(xs[e], E) - f) / np.linalg.norm(f)
                assert res < 1.05 * tol and rr5[e] < tol, (tol, E, res, rr5[e], its5[e])
                assert abs(res - rr5[e]) < 1e-3 * tol + 1e-2 * res, (res, rr5[e])
            if tol == 1e-8:
                assert all(b <= 1.5 * a + 10 for a, b in zip(its1, its5)), (its1, its5)
            print("tol", tol, "iterations FP64", its1, "mixed", its5)
    finally:
        S.soft_destroy(plan)


@pytest.mark.parametrize("contour", [S.CONTOUR_SECS, S.CONTOUR_TFECS, S.ABSORB_CAP, S.ABSORB_TFAP])
def test_pcg_contours_and_absorbers(contour):
    """The stationary solver on the smooth contours (Eqs. qSECS, qTFECS) and
    with the comparison absorbers (Sec. IV), banded preconditioner in FP64
    and the mixed mode: every residual recomputed by the oracle's A built
    with the same contour."""
    n, box, R0, th = 256, (-40.0, 40.0, -40.0, 40.0), 30.0, 0.4
    okind = {S.CONTOUR_SECS: T.SECS, S.CONTOUR_TFECS: T.TFECS, S.ABSORB_CAP: T.CAP,
             S.ABSORB_TFAP: T.TFAP}[contour]
    plan = S.soft_create((n, n), box, R0, th, 0.02, prec=S.SOFT_C128, soft_a2=1.0, contour=contour,
                         cap_energy=2.0, tfap_kmin=0.25)
    try:
        p2 = P.Problem2D(n, n, box, R0, theta=th, kind=okind, alpha=0.5, a2=1.0, dt=0.02, e_cap=2.0,
                         kmin=0.25)
        st = ST.Stationary2D(p2, nbw=10, kind=okind, R0=R0, theta=th)
        xg = -40.0 + 80.0 / n * (np.arange(n) + 0.5)
        f = -np.exp(-(xg[None, :] ** 2 + (xg[:, None] - 3.0) ** 2) / 32.0).astype(np.complex128)
        Es = [0.4, 1.3]
        out = torch.zeros((len(Es), n, n), dtype=torch.complex128, device="cuda")
        for pc in (1, 5):
            rc, its, rr = S.sse_pcg_solve(plan, Es, dev(f), out, tol=1e-8, maxit=3000, precond=pc)
            assert rc == 0, (pc, rc, its, rr)
            xs = host(out)
            for e, E in enumerate(Es):
                res = np.linalg.norm(st.apply_A(xs[e], E) - f) / np.linalg.norm(f)
                assert res < TRUE_RES_TOL, (pc, E, res, its[e])
            print("contour", contour, "precond", pc, "iterations", its)
    finally:
        S.soft_destroy(plan)


@pytest.mark.parametrize("precond", [0, 1])
def test_pcg_solves_batch_small(precond):
    """Four energies at once; each residual recomputed with the oracle's A
    (FP64 numpy) must meet the tolerance."""
    plan, p2, st = setup()
    try:
        n = 256
        xg = -40.0 + 80.0 / n * (np.arange(n) + 0.5)
        f = -np.exp(-(xg[None, :] ** 2 + (xg[:, None] - 3.0) ** 2) / 32.0).astype(np.complex128)
        Es = [0.2, 0.55, 1.1, 1.9]
        out = torch.zeros((len(Es), n, n), dtype=torch.complex128, device="cuda")
        rc, its, rr = S.sse_pcg_solve(plan, Es, dev(f), out, tol=1e-8, maxit=2000, precond=precond)
        assert rc == 0, (rc, its, rr)
        xs = host(out)
        for e, E in enumerate(Es):
            res = np.linalg.norm(st.apply_A(xs[e], E) - f) / np.linalg.norm(f)
            assert res < TRUE_RES_TOL, (E, res, its[e])
            assert rr[e] < 1e-8
        # the oracle's own COCG reaches the same solution
        xo, ito, _ = ST.cocg(lambda v: st.apply_A(v, Es[1]),
                             (lambda r: st.precond_simple(r, Es[1])) if precond == 0 else
                             (lambda r: st.precond_band(r, Es[1])), f, tol=1e-10, maxit=3000)
        assert relerr(xs[1], xo) < 1e-6
        print("iterations", its, "oracle", ito)
    finally:
        S.soft_destroy(plan)


def test_free_unscaled_problem_converges_in_one_iteration():
    """q = 1, U = 0: the simple preconditioner is A^-1 exactly (Eq. PreconFFT),
    so CG stops after one iteration; the banded one reduces to it."""
    plan, p2, st = setup(theta=0.0, charge=0.0)
    try:
        n = 256
        rng = np.random.default_rng(5)
        f = rng.standard_normal((n, n)) + 0j
        out = torch.zeros((1, n, n), dtype=torch.complex128, device="cuda")
        for pc in (0, 1):
            rc, its, rr = S.sse_pcg_solve(plan, [0.37], dev(f), out, tol=1e-10, maxit=50, precond=pc)
            assert rc == 0 and its[0] == 1 and rr[0] < 1e-10
    finally:
        S.soft_destroy(plan)


def test_bad_arguments_and_iteration_cap():
    plan, p2, st = setup()
    try:
        n = 256
        f = np.ones((n, n), dtype=np.complex128)
        out = torch.zeros((1, n, n), dtype=torch.complex128, device="cuda")
        with pytest.raises(S.SoftError):
            S.sse_pcg_solve(plan, [0.5], dev(f), out, tol=-1.0)
        with pytest.raises(S.SoftError):
            S.sse_pcg_solve(plan, [float("nan")], dev(f), out)
        rc, its, rr = S.sse_pcg_solve(plan, [0.5], dev(f), out, tol=1e-14, maxit=3, precond=0)
        assert rc == -5 and its[0] == 3 and rr[0] > 1e-14
    finally:
        S.soft_destroy(plan)


@pytest.mark.slow
def test_w4_full_size_sampled_energies():
    """The stationary workload at full size (1024^2, W3 box and contour,
    Gaussian source) with the banded preconditioner: four of its 64 energies
    in FP64 (precond 1) and FP32 (precond 4), all 64 in the mixed mode the
    benchmark times (precond 5); the residual of every returned solution is
    recomputed by the oracle's A."""
    w = W.w4()
    n = w["nx"]
    plan = S.soft_create((n, n), w["box"], w["R0"], w["theta"], 0.02, prec=S.SOFT_C128,
                         soft_a2=w["a2"])
    try:
        p2 = P.Problem2D(n, n, w["box"], w["R0"], theta=w["theta"], a2=w["a2"], dt=0.02)
        st = ST.Stationary2D(p2, nbw=10, kind=T.SHARP, R0=w["R0"], theta=w["theta"])
        for pc in (1, 4, 5):
            Es = list(w["E"]) if pc == 5 else list(w["E"][[0, 21, 42, 63]])
            out = torch.zeros((len(Es), n, n), dtype=torch.complex128, device="cuda")
            rc, its, rr = S.sse_pcg_solve(plan, Es, dev(w["f"]), out, tol=w["tol"], maxit=3000,
                                          precond=pc)
            assert rc == 0, (pc, rc, its, rr)
            xs = host(out)
            for e, E in enumerate(Es):
                res = np.linalg.norm(st.apply_A(xs[e], E) - w["f"]) / np.linalg.norm(w["f"])
                assert res < w["tol"] * (1 + 1e-4), (pc, E, res)
            print("W4 iterations (band, precond %d):" % pc, its)
    finally:
        S.soft_destroy(plan)
