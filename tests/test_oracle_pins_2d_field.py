"""Pins of the two oracle parts that the 1D pins leave open: the 2D step and
the laser-field coupling.

2D (Sec. II, the scheme after Eq. C_FD on a product grid; the paper's closing
remark of Sec. III that the method generalises to several dimensions): with
K = K_x + K_y, C = C_x (x) I + I (x) C_y and a separable potential
U = U_x(x) + U_y(y), every factor of one step is a Kronecker product, so a
product state phi(x) chi(y) must stay the product of the two 1D oracle runs.
The grids are not square and the two axes differ in box, strip and
potential, so a step that swapped the axes, used one axis's C or k on the
other, or dropped C_y would fail.

Field (the laser coupling U_L = E(t) x of the length gauge, taken at
t + tau/2 as Sec. II prescribes for U(x, t)): with theta = 0, U0 = 0 and the
packet far from the strips, i dpsi/dt = [-1/2 d^2/dx^2 + E(t) x] psi has the
closed form psi(x, t) = exp(i b x - i g) psi_free(x - c, t) with
b = -int E, c = int b, g = int b^2/2 (all from 0 to t).  Strang splitting
with the field at the midpoint is second order in tau against it; a flipped
sign of E x misses it by O(1) and a field taken at t instead of t + tau/2
is only first order, which the test shows on the same closed form."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import propagate as P
from oracle import tables as T


def free_packet(x, t, sigma, x0, k0, L=None, images=0):
    """Free Gaussian, i dpsi/dt = -1/2 psi'', initially
    (pi sigma^2)^{-1/4} exp(-(x - x0)^2/(2 sigma^2) + i k0 x), summed over
    `images` periodic images of a box of length L."""
    s2 = sigma * sigma
    out = 0
    for m in range(-images, images + 1):
        xx = x + (m * L if images else 0.0)
        out = out + ((s2 / math.pi) ** 0.25 * (s2 + 1j * t) ** -0.5
                     * np.exp(-(xx - x0 - k0 * t) ** 2 / (2 * (s2 + 1j * t))
                              + 1j * k0 * (xx - x0) - 0.5j * k0 * k0 * t + 1j * k0 * x0))
    return out


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ 2D ----
def _separable_case(kind, theta):
    nx, ny = 128, 64
    box = (-20.0, 20.0, -12.0, 12.0)
    R0 = 9.0
    dt = 0.02
    p2 = P.Problem2D(nx, ny, box, R0, theta=theta, kind=kind, dt=dt, potential=False)
    px = P.Problem1D(nx, box[0], box[1], R0, theta=theta, kind=kind, dt=dt, potential=False)
    py = P.Problem1D(ny, box[2], box[3], R0, theta=theta, kind=kind, dt=dt, potential=False)
    zx = T.z_contour(px.x, kind, R0, box[1], theta)
    zy = T.z_contour(py.x, kind, R0, box[3], theta)
    Ux = T.soft_coulomb([zx], 2.0, 1.0)                     # complex on the scaled strip
    Uy = 0.02 * zy ** 2 - 0.3 * T.soft_coulomb([zy], 1.0, 1.0)
    px.U0, py.U0 = Ux, Uy
    p2.U = np.ascontiguousarray(Uy[:, None] + Ux[None, :])
    phi = free_packet(px.x, 0.0, 1.5, 2.0, 1.3)
    chi = free_packet(py.x, 0.0, 1.0, -1.0, -0.8)
    return p2, px, py, phi, chi


@pytest.mark.parametrize("kind,theta", [(T.SHARP, 0.5), (T.SECS, 0.6)])
def test_2d_step_is_the_product_of_two_1d_steps(kind, theta):
    """One 2D step on a product state with a separable potential equals the
    outer product of the 1D oracle steps of each axis, over 40 steps, to
    round-off (the state reaches both strips)."""
    p2, px, py, phi, chi = _separable_case(kind, theta)
    nst = 40
    got = p2.step(chi[:, None] * phi[None, :], nst)
    ref = py.step(chi, nst)[:, None] * px.step(phi, nst)[None, :]
    assert np.abs(p2.Cx[1]).max() > 0 and np.abs(p2.Cy[1]).max() > 0
    assert relerr(got, ref) < 1e-13
    # the two axes are not interchangeable here: the y factor stepped on the
    # x axis's box (another h, k grid and strip) is far from it
    swapped = P.Problem1D(64, -20.0, 20.0, 9.0, theta=theta, kind=kind, dt=0.02, potential=False)
    swapped.U0 = py.U0
    assert relerr(swapped.step(chi, nst), py.step(chi, nst)) > 1e-3


def test_2d_free_gaussian_closed_form():
    """theta = 0, U = 0 on a non-square grid: C = 0 and the 2D scheme must
    give the product of the two closed-form free Gaussians, summed over the
    periodic images of each axis, after 400 steps."""
    nx, ny = 256, 128
    box = (-40.0, 40.0, -25.0, 25.0)
    dt, nst = 0.05, 400
    p2 = P.Problem2D(nx, ny, box, 30.0, theta=0.0, dt=dt, potential=False)
    x, y = p2.x, p2.y
    Lx, Ly = box[1] - box[0], box[3] - box[2]
    fx = lambda t: free_packet(x, t, 2.5, -4.0, 0.9, Lx, 3)
    fy = lambda t: free_packet(y, t, 1.8, 3.0, -0.6, Ly, 3)
    got = p2.step(fy(0.0)[:, None] * fx(0.0)[None, :], nst)
    t = nst * dt
    ex = fy(t)[:, None] * fx(t)[None, :]
    assert relerr(got, ex) < 1e-11


# --------------------------------------------------------------- field ----
E0, OMEGA, NCYC = 0.2, 0.5, 2.0
TPULSE = NCYC * 2 * math.pi / OMEGA


def _kick_integrals(t):
    """b = -int_0^t E, c = int_0^t b, g = int_0^t b^2/2 by adaptive
    quadrature (a library routine) of the pulse E0 sin^2(pi s/T) sin(omega s)."""
    E = lambda s: float(T.field_E(s, E0, OMEGA, NCYC))
    b = lambda s: -quad(E, 0.0, s, epsabs=1e-14, epsrel=1e-13, limit=400)[0]
    c = quad(b, 0.0, t, epsabs=1e-14, epsrel=1e-12, limit=400)[0]
    g = quad(lambda s: 0.5 * b(s) ** 2, 0.0, t, epsabs=1e-14, epsrel=1e-12, limit=400)[0]
    return b(t), c, g


@pytest.fixture(scope="module")
def field_case():
    n, a, bb = 2048, -160.0, 160.0
    sig, x0, k0 = 2.0, -3.0, 0.4
    tend = 0.6 * TPULSE                    # E(tend) != 0: the midpoint rule matters here
    x, _ = T.grid(n, a, bb)
    b, c, g = _kick_integrals(tend)
    exact = np.exp(1j * b * x - 1j * g) * free_packet(x - c, tend, sig, x0, k0)
    psi0 = free_packet(x, 0.0, sig, x0, k0)

    def run(nst, sign=1.0, t0=0.0):
        p = P.Problem1D(n, a, bb, R0=150.0, theta=0.0, dt=tend / nst, potential=False)
        return relerr(p.step(psi0, nst, t0=t0 * p.dt, field=(sign * E0, OMEGA, NCYC)), exact)
    return run


def test_field_matches_the_uniform_field_closed_form_to_second_order(field_case):
    errs = [field_case(nst) for nst in (250, 500, 1000)]
    assert errs[-1] < 3e-6
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


def test_field_pin_detects_a_flipped_sign_and_a_field_taken_at_t(field_case):
    """The same closed form rejects E x with the wrong sign (an O(1) error)
    and the field evaluated at the start of each step instead of its
    midpoint (started half a step early: first order, 2x per halving)."""
    assert field_case(1000, sign=-1.0) > 0.5
    at_t = [field_case(nst, t0=-0.5) for nst in (250, 500)]
    assert at_t[1] > 1e-3 and 1.8 < at_t[0] / at_t[1] < 2.2


def test_secs_contour_at_zero_angle_is_unscaled():
    """Eq. qSECS with theta = 0 gives q = 1 everywhere, so z(x) = x, C = 0 and
    the step must equal the unscaled one (the closed form of z divides by
    theta and needs the limit)."""
    n, a, b, R0 = 256, -20.0, 20.0, 15.0
    x, _ = T.grid(n, a, b)
    assert np.array_equal(T.z_contour(x, T.SECS, R0, b, 0.0), x.astype(np.complex128))
    ps = P.Problem1D(n, a, b, R0, theta=0.0, kind=T.SECS, dt=0.02)
    p0 = P.Problem1D(n, a, b, R0, theta=0.0, kind=T.SHARP, dt=0.02)
    assert max(np.abs(ps.Cd).max(), np.abs(ps.Cs).max()) == 0.0
    psi0 = free_packet(x, 0.0, 1.5, 3.0, 0.8)
    assert relerr(ps.step(psi0, 50), p0.step(psi0, 50)) < 1e-14
