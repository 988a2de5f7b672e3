"""Pins of the 3D oracle step (the scheme after Eq. C_FD of Sec. II on a
product grid; the multidimensional case named at the end of Sec. V).

With K = K_x + K_y + K_z, C = C_x + C_y + C_z as Kronecker sums and a
potential that splits across the axes, every factor of one step is a
Kronecker product, so a product state must stay the product of the lower-
dimensional oracle runs:
  - U = U_x(x) + U_y(y) + U_z(z): the product of three 1D steps;
  - U = U_xy(x, y) + U_z(z) with a non-separable U_xy: the 2D step (pinned
    on its own) times the 1D step along z.
The three axes differ in length, box, strip and potential, so a step that
permuted the axes, used one axis's C or k on another, or dropped one axis's
CN would fail.  At theta = 0 with U = 0 the 3D free Gaussian is the product
of three closed forms summed over each axis's periodic images."""
import numpy as np
import pytest

from oracle import propagate as P
from oracle import tables as T

from test_oracle_pins_2d_field import free_packet, relerr

NX, NY, NZ = 64, 32, 16
BOX = (-20.0, 20.0, -12.0, 12.0, -8.0, 8.0)


def _axis(n, a, b, r0, kind, theta, dt):
    return P.Problem1D(n, a, b, r0, theta=theta, kind=kind, dt=dt, potential=False)


def _case(kind, theta):
    """The 3D problem with the SAME R0 on every axis (the 3D plan takes one
    R0); the per-axis 1D problems built from it."""
    dt = 0.02
    r0 = 5.0
    p3 = P.Problem3D((NX, NY, NZ), BOX, r0, theta=theta, kind=kind, dt=dt, potential=False)
    px = _axis(NX, BOX[0], BOX[1], r0, kind, theta, dt)
    py = _axis(NY, BOX[2], BOX[3], r0, kind, theta, dt)
    pz = _axis(NZ, BOX[4], BOX[5], r0, kind, theta, dt)
    return p3, px, py, pz


@pytest.mark.parametrize("kind,theta", [(T.SHARP, 0.5), (T.SECS, 0.6)])
def test_3d_step_is_the_product_of_three_1d_steps(kind, theta):
    p3, px, py, pz = _case(kind, theta)
    zx = T.z_contour(px.x, kind, 5.0, BOX[1], theta)
    zy = T.z_contour(py.x, kind, 5.0, BOX[3], theta)
    zz = T.z_contour(pz.x, kind, 5.0, BOX[5], theta)
    px.U0 = T.soft_coulomb([zx], 2.0, 1.0)
    py.U0 = 0.02 * zy ** 2 - 0.3 * T.soft_coulomb([zy], 1.0, 1.0)
    pz.U0 = -0.5 * T.soft_coulomb([zz], 0.5, 1.0) + 0.01 * zz
    p3.U = np.ascontiguousarray(pz.U0[:, None, None] + py.U0[None, :, None] + px.U0[None, None, :])
    fx = free_packet(px.x, 0.0, 1.5, 2.0, 1.3)
    fy = free_packet(py.x, 0.0, 1.0, -1.0, -0.8)
    fz = free_packet(pz.x, 0.0, 0.8, 0.5, 1.1)
    nst = 30
    got = p3.step(fz[:, None, None] * fy[None, :, None] * fx[None, None, :], nst)
    ref = (pz.step(fz, nst)[:, None, None] * py.step(fy, nst)[None, :, None]
           * px.step(fx, nst)[None, None, :])
    for c in p3.C:
        assert np.abs(c[1]).max() > 0                  # every axis has a strip
    assert relerr(got, ref) < 1e-13


def test_3d_step_is_the_2d_step_times_the_1d_step():
    """A non-separable U_xy plus U_z: the 3D step equals the (separately
    pinned) 2D step on (x, y) times the 1D step along z."""
    kind, theta, dt = T.SECS, 0.5, 0.02
    p3, _, _, pz = _case(kind, theta)
    p2 = P.Problem2D(NX, NY, BOX[:4], 5.0, theta=theta, kind=kind, dt=dt, a2=1.5)
    zz = T.z_contour(pz.x, kind, 5.0, BOX[5], theta)
    pz.U0 = 0.03 * zz ** 2
    p3.U = np.ascontiguousarray(p2.U[None, :, :] + pz.U0[:, None, None])
    x, y = p2.x, p2.y
    g2 = (free_packet(y, 0.0, 1.2, 0.5, 0.4)[:, None] * free_packet(x, 0.0, 2.0, -1.0, 0.7)[None, :]
          + 0.5 * free_packet(y, 0.0, 0.9, -2.0, -0.3)[:, None] * free_packet(x, 0.0, 1.1, 3.0, 0.0)[None, :])
    gz = free_packet(pz.x, 0.0, 0.9, -0.5, 0.6)
    nst = 25
    got = p3.step(gz[:, None, None] * g2[None, :, :], nst)
    ref = pz.step(gz, nst)[:, None, None] * p2.step(g2, nst)[None, :, :]
    assert relerr(got, ref) < 1e-13


def test_3d_free_gaussian_closed_form():
    """theta = 0, U = 0: C = 0 and the scheme gives the product of three
    closed-form free Gaussians, each summed over its axis's periodic images,
    after 200 steps."""
    n = (64, 32, 32)                    # h = 0.75: the packets are band-limited to 1e-13
    box = (-24.0, 24.0, -12.0, 12.0, -12.0, 12.0)
    dt, nst = 0.05, 200
    p3 = P.Problem3D(n, box, 9.0, theta=0.0, dt=dt, potential=False)
    L = [box[2 * d + 1] - box[2 * d] for d in range(3)]
    f = [lambda t: free_packet(p3.x[0], t, 2.5, -4.0, 0.9, L[0], 3),
         lambda t: free_packet(p3.x[1], t, 2.2, 3.0, -0.6, L[1], 3),
         lambda t: free_packet(p3.x[2], t, 2.3, 1.0, 0.5, L[2], 3)]
    prod = lambda t: f[2](t)[:, None, None] * f[1](t)[None, :, None] * f[0](t)[None, None, :]
    got = p3.step(prod(0.0), nst)
    assert relerr(got, prod(nst * dt)) < 1e-11
