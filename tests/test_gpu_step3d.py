"""GPU parity of the 3D ECS split-operator step (the scheme after Eq. C_FD of
Sec. II with K = K_x + K_y + K_z and C = C_x + C_y + C_z as Kronecker sums;
the multidimensional case named at the end of Sec. V) against the oracle's
literal 4-FFT 3D step.  complex128: rel-L2 <= 1e-11; complex64: 1e-5."""
import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1505_06707_gb300 as S  # noqa: E402
import workloads as W  # noqa: E402
from oracle import propagate as P  # noqa: E402
from oracle import tables as T  # noqa: E402

CT = {S.SOFT_C64: torch.complex64, S.SOFT_C128: torch.complex128}


def tol(prec):
    return 1e-11 if prec == S.SOFT_C128 else 1e-5


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run3d(n, box, R0, theta, dt, psi0, nsteps, prec, calls=1, **opt):
    plan = S.soft_create(tuple(n), box, R0, theta, dt, prec=prec, **opt)
    try:
        d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
        t = 0.0
        for c in range(calls):
            t = S.soft_step(plan, d, nsteps // calls, t)
        torch.cuda.synchronize()
        assert abs(t - (nsteps // calls) * calls * dt) < 1e-9
        return d.cpu().numpy().astype(np.complex128), S.soft_last_launches(plan)
    finally:
        S.soft_destroy(plan)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    S.load()


# non-cubic grid, every axis with its own length, box and strip block
CASE = dict(n=(256, 64, 128), box=(-20.0, 20.0, -16.0, 16.0, -24.0, 24.0), R0=12.0)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("kind,theta", [(T.SHARP, 0.4), (T.SECS, 0.6), (T.TFECS, 0.0)])
def test_step3d_matches_oracle(prec, kind, theta):
    """20 steps in two calls (graph replay of 8-step chunks plus a remainder)
    on the soft-Coulomb potential: every element against the oracle."""
    n, box, R0 = CASE["n"], CASE["box"], CASE["R0"]
    dt = 0.02
    psi0 = W.w6_state(n, box, seed=5, noise=1e-3)
    ref = P.Problem3D(n, box, R0, theta=theta, kind=kind, dt=dt, a2=1.0)
    assert all(np.abs(c[1]).max() > 0 for c in ref.C)          # strips on all axes
    exp = ref.step(ref.step(psi0, 10), 10)
    got, launches = run3d(n, box, R0, theta, dt, psi0, 20, prec, calls=2, contour=kind, soft_a2=1.0)
    assert launches > 0
    assert relerr(got, exp) < tol(prec)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("kind,theta", [(T.SECS, 0.5), (T.TFAP, 0.0)])
def test_step3d_smallest_axes(prec, kind, theta):
    """64-point axes (the smallest 3D size, radix-2 passes): with SECS every
    axis has a strip; with the TFAP comparison absorber none has (C = 0), so
    every row is a full row pass.  9 steps (one graph chunk and the last)."""
    n, box, R0 = (64, 64, 64), (-16.0, 16.0, -16.0, 16.0, -16.0, 16.0), 10.0
    dt = 0.02
    psi0 = W.w6_state(n, box, seed=9, noise=1e-3)
    ref = P.Problem3D(n, box, R0, theta=theta, kind=kind, dt=dt, a2=1.0)
    exp = ref.step(psi0, 9)
    got, _ = run3d(n, box, R0, theta, dt, psi0, 9, prec, contour=kind, soft_a2=1.0)
    assert relerr(got, exp) < tol(prec)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_step3d_wide_y_strip(prec):
    """A long y axis with a wide strip block (320 of 512 rows): the y-strip
    CN pass takes its narrowest tile (32 lines per CTA) and its longest
    sweeps; 10 steps against the oracle."""
    n, box, R0 = (64, 512, 64), (-16.0, 16.0, -32.0, 32.0, -16.0, 16.0), 12.0
    dt = 0.02
    psi0 = W.w6_state(n, box, seed=13, noise=1e-3)
    ref = P.Problem3D(n, box, R0, theta=0.5, kind=T.SECS, dt=dt, a2=1.0)
    assert int((np.abs(ref.C[1][1]) > 0).sum()) >= 300
    exp = ref.step(psi0, 10)
    got, _ = run3d(n, box, R0, 0.5, dt, psi0, 10, prec, contour=T.SECS, soft_a2=1.0)
    assert relerr(got, exp) < tol(prec)


def test_step3d_free_gaussian_closed_form():
    """theta = 0, U = 0: the product of three closed-form free Gaussians
    summed over the periodic images of each axis (200 steps, complex128)."""
    from test_oracle_pins_2d_field import free_packet
    n = (128, 64, 64)                   # h = 0.75: band-limited packets
    box = (-48.0, 48.0, -24.0, 24.0, -24.0, 24.0)
    dt, nst = 0.05, 200
    x = [T.grid(n[d], box[2 * d], box[2 * d + 1])[0] for d in range(3)]
    L = [box[2 * d + 1] - box[2 * d] for d in range(3)]
    prm = [(2.5, -4.0, 0.9), (2.2, 3.0, -0.6), (2.3, 1.0, 0.5)]

    def prod(t):
        f = [free_packet(x[d], t, *prm[d], L[d], 3) for d in range(3)]
        return f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    got, _ = run3d(n, box, 9.0, 0.0, dt, prod(0.0), nst, S.SOFT_C128, charge=0.0)
    assert relerr(got, prod(nst * dt)) < 1e-11


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_set_potential_3d(prec):
    """soft_set_potential on a 3D plan after a first call captured the step
    graph: the replayed graph must use the rewritten table (an anisotropic
    well at the complex coordinates, 16 + 16 steps against the oracle)."""
    n, box, R0, th = CASE["n"], CASE["box"], CASE["R0"], 0.4
    dt = 0.02
    ref = P.Problem3D(n, box, R0, theta=th, dt=dt, a2=1.0)
    z = [T.z_contour(ref.x[d], T.SHARP, R0, box[2 * d + 1], th, 0.5) for d in range(3)]
    U = -2.0 * np.exp(-(z[0][None, None, :] ** 2 + 0.5 * z[1][None, :, None] ** 2
                        + 0.25 * z[2][:, None, None] ** 2) / 9.0)
    psi0 = W.w6_state(n, box, seed=11, noise=1e-3)
    plan = S.soft_create(n, box, R0, th, dt, prec=prec, soft_a2=1.0)
    try:
        d = torch.tensor(psi0, dtype=CT[prec], device="cuda")
        t = S.soft_step(plan, d, 16, 0.0)
        S.soft_set_potential(plan, U.ravel())
        S.soft_step(plan, d, 16, t)
        torch.cuda.synchronize()
        got = d.cpu().numpy().astype(np.complex128)
    finally:
        S.soft_destroy(plan)
    mid = ref.step(psi0, 16)
    ref.U = np.ascontiguousarray(U)
    assert relerr(got, ref.step(mid, 16)) < tol(prec)


@pytest.fixture(scope="module")
def w6_case():
    cfg = W.w6()
    psi0 = W.w6_state(cfg["n"], cfg["box"], seed=0)
    ref = P.Problem3D(cfg["n"], cfg["box"], cfg["R0"], theta=cfg["theta"], kind=cfg["kind"],
                      dt=cfg["dt"], a2=cfg["a2"])
    return cfg, psi0, ref.step(psi0, 10)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_w6_full_size_few_steps(prec, w6_case):
    """The benchmark's 3D workload at full size (256^3), 10 steps (one
    8-step graph replay between the first and last step) in the launch
    configuration the benchmark times, every element against the oracle."""
    cfg, psi0, exp = w6_case
    got, _ = run3d(cfg["n"], cfg["box"], cfg["R0"], cfg["theta"], cfg["dt"], psi0, 10, prec,
                   contour=cfg["kind"], soft_a2=cfg["a2"])
    assert relerr(got, exp) < tol(prec)


def test_step3d_rejects_bad_grids():
    box = (-16.0, 16.0, -16.0, 16.0, -16.0, 16.0)
    for n in [(32, 64, 64), (64, 64, 4096), (100, 64, 64)]:
        with pytest.raises(S.SoftError):
            S.soft_create(n, box, 8.0, 0.4, 0.02, prec=S.SOFT_C64)
    with pytest.raises(ValueError):
        S.soft_create((64, 64, 64), box[:4], 8.0, 0.4, 0.02, prec=S.SOFT_C64)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("nsteps", [0, 1, 2, 3, 10, 11])
def test_call_lengths_3d(nsteps, prec):
    """Calls of 0 (no-op), 1 (the first step is also the last), 2 (no middle
    steps), 3, 10 and 11 steps (an 8-step graph replay plus a remainder)
    against the oracle."""
    n, box, R0 = (128, 64, 64), (-20.0, 20.0, -16.0, 16.0, -16.0, 16.0), 10.0
    psi0 = W.w6_state(n, box, seed=17, noise=1e-3)
    ref = P.Problem3D(n, box, R0, theta=0.5, kind=T.SECS, dt=0.02, a2=1.0).step(psi0, nsteps)
    got, launches = run3d(n, box, R0, 0.5, 0.02, psi0, nsteps, prec, contour=T.SECS, soft_a2=1.0)
    if nsteps == 0:
        assert launches == 0
        assert np.array_equal(got, psi0.astype(np.complex64 if prec == S.SOFT_C64 else np.complex128))
    else:
        assert launches == 4 * nsteps + 3               # 4 passes per step, K_y/2, K_z/2, K_x/2
        assert relerr(got, ref) < tol(prec)


@functools.lru_cache(maxsize=None)
def longest_axis_case(axis):
    n = [64, 64, 64]
    n[axis] = 2048
    n = tuple(n)
    box = (-16.0, 16.0) * 3
    psi0 = W.w6_state(n, box, seed=19 + axis, noise=1e-3)
    ref = P.Problem3D(n, box, 13.0, theta=0.5, kind=T.SECS, dt=0.02, a2=1.0)
    assert int((np.abs(ref.C[axis][1]) > 0).sum()) >= 380
    return n, box, psi0, ref.step(psi0, 6)


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_step3d_longest_axis(axis, prec):
    """One axis of 2048 points (the longest the 3D plan takes) with two of
    64 in one box [-16, 16]^3: the x row pass, the y-strip CN pass and the y
    lines, or the z lines, at their longest.  SECS theta = 0.5 from R0 = 13
    puts a 386-row strip block on the long axis (h = 1/64; for complex128
    on y that is near the y-strip pass's shared-memory limit) and a 14-row
    one on the short axes (h = 1/2); 6 steps against the oracle."""
    n, box, psi0, exp = longest_axis_case(axis)
    got, launches = run3d(n, box, 13.0, 0.5, 0.02, psi0, 6, prec, contour=T.SECS, soft_a2=1.0)
    assert launches == 4 * 6 + 3
    assert relerr(got, exp) < tol(prec)
