"""GPU parity of the 2D ECS split-operator step (Sec. II with separable K and
C = C_x (x) I + I (x) C_y) against the oracle's literal 4-FFT 2D step.
complex128: rel-L2 <= 1e-11.  complex64: 1e-5, the FP32 target."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1505_06707_gb300 as S  # noqa: E402
import workloads as W  # noqa: E402
from oracle import propagate as P  # noqa: E402
from oracle import tables as T  # noqa: E402

CT = {S.SOFT_C64: torch.complex64, S.SOFT_C128: torch.complex128}


def tol(prec, nsteps=None, n=None):
    return 1e-11 if prec == S.SOFT_C128 else 1e-5


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run2d(nx, ny, box, R0, theta, dt, psi0, nsteps, prec, **opt):
    plan = S.soft_create((nx, ny), box, R0, theta, dt, prec=prec, **opt)
    try:
        d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
        t = S.soft_step(plan, d, nsteps, 0.0)
        torch.cuda.synchronize()
        assert abs(t - nsteps * dt) < 1e-9
        launches = S.soft_last_launches(plan)
        return d.cpu().numpy().astype(np.complex128), launches
    finally:
        S.soft_destroy(plan)


def packet2d(nx, ny, box, seed):
    rng = np.random.default_rng(seed)
    x = box[0] + (box[1] - box[0]) / nx * (np.arange(nx) + 0.5)
    y = box[2] + (box[3] - box[2]) / ny * (np.arange(ny) + 0.5)
    psi = np.zeros((ny, nx), dtype=np.complex128)
    for _ in range(3):
        cx, cy = rng.uniform(-0.5, 0.5, 2) * box[1]
        kx, ky = rng.uniform(-1.5, 1.5, 2)
        s = rng.uniform(2.0, 4.0)
        psi += np.exp(-((y[:, None] - cy) ** 2 + (x[None, :] - cx) ** 2) / (2 * s * s)
                      + 1j * (kx * x[None, :] + ky * y[:, None]))
    # a small random component reaches every mode, including the strips
    psi += 1e-3 * (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx)))
    return psi


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    S.load()


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_set_potential_2d(prec):
    """soft_set_potential on a 2D plan: an anisotropic well at (z(x), z(y))
    replaces the soft-Coulomb potential after a first call has captured the
    step graph; the replayed graph must use the rewritten tables (oracle with
    the same U, 24 steps)."""
    n, box, R0, th = 256, (-40.0, 40.0, -40.0, 40.0), 30.0, 0.4
    ref = P.Problem2D(n, n, box, R0, theta=th, a2=1.0, dt=0.02)
    zx = T.z_contour(ref.x, T.SHARP, R0, box[1], th, 0.5)
    zy = T.z_contour(ref.y, T.SHARP, R0, box[3], th, 0.5)
    U = -2.0 * np.exp(-(zx[None, :] ** 2 + 0.5 * zy[:, None] ** 2) / 9.0)
    psi0 = packet2d(n, n, box, 99)
    plan = S.soft_create((n, n), box, R0, th, 0.02, prec=prec, soft_a2=1.0)
    try:
        d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
        S.soft_step(plan, d, 24, 0.0)
        S.soft_set_potential(plan, U)
        d.copy_(torch.tensor(psi0, dtype=CT[prec]))
        S.soft_step(plan, d, 24, 0.0)
        torch.cuda.synchronize()
        ref.U = np.ascontiguousarray(U, dtype=np.complex128)
        want = ref.step(psi0, 24)
        assert relerr(d.cpu().numpy().astype(np.complex128), want) < tol(prec, 24, n)
    finally:
        S.soft_destroy(plan)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("shape", [(256, 256), (512, 256), (256, 512)])
def test_small_grids_match_oracle(shape, prec):
    """Square and non-square grids (the same box, so h differs per axis),
    sharp ECS theta = 0.4 on both axes, soft-Coulomb a^2 = 1; 40 steps
    (exercises the captured-graph path)."""
    nx, ny = shape
    box = (-40.0, 40.0, -40.0, 40.0)
    R0 = 30.0
    psi0 = packet2d(nx, ny, box, nx + 7 * ny)
    ref = P.Problem2D(nx, ny, box, R0, theta=0.4, a2=1.0, dt=0.02).step(psi0, 40)
    got, launches = run2d(nx, ny, box, R0, 0.4, 0.02, psi0, 40, prec, soft_a2=1.0)
    assert relerr(got, ref) < tol(prec, 40, max(nx, ny))
    assert launches == 2 * 40 + 2            # a row and a column pass per step, K_y/2 and K_x/2


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("kind", [S.ABSORB_CAP, S.ABSORB_TFAP])
def test_comparison_absorbers_2d(kind, prec):
    """The Sec. IV comparison absorbers on both axes, U_a(x) + U_a(y) on a
    real contour (no strips): 256^2, 40 steps."""
    from oracle import tables as T
    n = 256
    box = (-40.0, 40.0, -40.0, 40.0)
    R0 = 30.0
    psi0 = packet2d(n, n, box, 31 + kind)
    okind = T.CAP if kind == S.ABSORB_CAP else T.TFAP
    ref = P.Problem2D(n, n, box, R0, theta=0.4, kind=okind, a2=1.0, dt=0.02, e_cap=2.0,
                      kmin=0.25).step(psi0, 40)
    got, _ = run2d(n, n, box, R0, 0.4, 0.02, psi0, 40, prec, soft_a2=1.0, contour=kind,
                   cap_energy=2.0, tfap_kmin=0.25)
    assert relerr(got, ref) < tol(prec, 40, n)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("contour", [S.CONTOUR_SECS, S.CONTOUR_TFECS])
def test_smooth_contours_2d(contour, prec):
    """SECS and TFECS (Eqs. qSECS, qTFECS) on both axes: 256^2, 40 steps
    against the oracle with the same contour."""
    n = 256
    box = (-40.0, 40.0, -40.0, 40.0)
    R0, th = 30.0, 0.4
    psi0 = packet2d(n, n, box, 41 + contour)
    okind = T.SECS if contour == S.CONTOUR_SECS else T.TFECS
    ref = P.Problem2D(n, n, box, R0, theta=th, kind=okind, alpha=0.5, a2=1.0, dt=0.02).step(psi0, 40)
    got, _ = run2d(n, n, box, R0, th, 0.02, psi0, 40, prec, soft_a2=1.0, contour=contour)
    assert relerr(got, ref) < tol(prec, 40, n)


def test_free_gaussian_closed_form_2d():
    """theta = 0, U = 0: the 2D step must reproduce the separable closed-form
    free Gaussian (summed over periodic images)."""
    n, b = 256, 40.0
    x = -b + 2 * b / n * (np.arange(n) + 0.5)
    L = 2 * b

    def free1(t, k0, s2=4.0):
        out = 0
        for m in range(-3, 4):
            xx = x + m * L
            out = out + ((s2 / math.pi) ** 0.25 * (s2 + 1j * t) ** -0.5
                         * np.exp(-(xx - k0 * t) ** 2 / (2 * (s2 + 1j * t)) + 1j * k0 * xx
                                  - 0.5j * k0 * k0 * t))
        return out
    psi0 = free1(0.0, 0.7)[None, :] * free1(0.0, -0.4)[:, None]
    got, _ = run2d(n, n, (-b, b, -b, b), 30.0, 0.0, 0.02, psi0, 50, S.SOFT_C128, charge=0.0)
    ref = free1(1.0, 0.7)[None, :] * free1(1.0, -0.4)[:, None]
    assert relerr(got, ref) < 1e-11


@pytest.mark.slow
@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_w3_full_size_few_steps(prec):
    """The 2D workload at full size (2048^2, [-200,200]^2, sharp theta = 0.4,
    four seeded Gaussians) for 6 steps, the same launch configuration the
    2D benchmark times, compared point by point with the oracle."""
    w = W.w3()
    nst = 6
    ref = P.Problem2D(w["nx"], w["ny"], w["box"], w["R0"], theta=w["theta"], a2=w["a2"],
                      dt=w["dt"]).step(w["psi0"], nst)
    got, _ = run2d(w["nx"], w["ny"], w["box"], w["R0"], w["theta"], w["dt"], w["psi0"], nst,
                   prec, soft_a2=w["a2"])
    assert relerr(got, ref) < tol(prec, nst, w["nx"])


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("nsteps", [0, 1, 2, 3, 17, 18])
def test_call_lengths_2d(nsteps, prec):
    """Calls of 0 (no-op), 1 (the first step is also the last: both half
    kinetic factors in one step), 2 (no middle steps), 3, 17 and 18 steps
    (a 16-step graph replay plus a remainder) against the oracle."""
    nx, ny = 256, 512
    box = (-40.0, 40.0, -40.0, 40.0)
    psi0 = packet2d(nx, ny, box, 21)
    ref = P.Problem2D(nx, ny, box, 30.0, theta=0.4, a2=1.0, dt=0.02).step(psi0, nsteps)
    got, launches = run2d(nx, ny, box, 30.0, 0.4, 0.02, psi0, nsteps, prec, soft_a2=1.0)
    assert launches == (2 * nsteps + 2 if nsteps else 0)
    if nsteps == 0:
        assert np.array_equal(got, psi0.astype(np.complex64 if prec == S.SOFT_C64 else np.complex128))
    else:
        assert relerr(got, ref) < tol(prec)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("shape", [(1024, 256), (256, 1024), (2048, 256), (256, 2048)])
def test_axis_lengths_2d(shape, prec):
    """Axes of 1024 and 2048 points beside a 256-point axis (the row and
    column kernels of the longest lines with the shortest), one box, so h
    differs fourfold or eightfold between the axes; SECS theta = 0.5 from
    R0 = 32 (a 410-row strip block on a 2048-point axis); 20 steps (a
    16-step graph replay) against the oracle."""
    nx, ny = shape
    box = (-40.0, 40.0, -40.0, 40.0)
    psi0 = packet2d(nx, ny, box, 3 * nx + ny)
    ref = P.Problem2D(nx, ny, box, 32.0, theta=0.5, kind=T.SECS, a2=1.0, dt=0.02)
    exp = ref.step(psi0, 20)
    got, launches = run2d(nx, ny, box, 32.0, 0.5, 0.02, psi0, 20, prec, contour=T.SECS, soft_a2=1.0)
    assert launches == 2 * 20 + 2
    assert relerr(got, exp) < tol(prec)
