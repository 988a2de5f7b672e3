"""Pins of the stationary-equation oracle (Sec. III) against definitions,
dense linear algebra and the special cases where the preconditioners are
exact."""
import json
import os

import numpy as np
import pytest

from oracle import propagate as P
from oracle import stationary as S
from oracle import tables as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_band_split_rule_n1024():
    """Sec. III (paragraph after Fig. 1): singletons k_1 and k_{N/2+1}, bands
    of N_BW = 10 and two mirror end bands of width in [N_BW, 2 N_BW - 1] next
    to the Nyquist index.  For N = 1024: 511 positive modes = 50 x 10 + 11."""
    g = json.load(open(os.path.join(GOLD, "paper_test_setup.json")))
    n, nbw = g["N"], g["N_BW"]
    bands = S.band_split(n, nbw)
    widths = [w for _, w in bands]
    assert bands[0] == (0, 1) and (n // 2, 1) in bands
    assert sum(widths) == n
    starts = [m for m, _ in bands]
    assert starts == sorted(starts)
    assert widths.count(11) == 2 and widths.count(10) == 100 and widths.count(1) == 2
    # the 11-wide bands touch the Nyquist index
    i = bands.index((n // 2, 1))
    assert widths[i - 1] == 11 and widths[i + 1] == 11


def _small(n=48, theta=0.5, kind=T.SHARP, potential=True):
    return P.Problem1D(n, -24.0, 24.0, R0=16.0, theta=theta, kind=kind, potential=potential)


def test_dense_A_is_complex_symmetric_and_matches_fft_apply():
    """A = F^-1 K F + C + U - E (Sec. III) is complex symmetric (the property
    that allows CG, Sec. III after Eq. linsys); its FFT application equals the
    dense product with F_{nj} = e^{i k_n x_j}/sqrt N (Eq. Fmatrix)."""
    st = S.Stationary1D(_small())
    A = st.dense_A(0.8)
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    v = np.random.default_rng(3).standard_normal(48) * (1 + 0.5j)
    assert np.abs(A @ v - st.apply_A(v, 0.8)).max() < 1e-12 * np.abs(A).max() * np.abs(v).max()


def test_X_complex_orthogonal_and_P_symmetric():
    """X^-1 = X^T (Sec. III after Eq. K_l) and P^-1 symmetric."""
    st = S.Stationary1D(_small(64))
    X, lam = st.dense_X()
    assert np.abs(X.T @ X - np.eye(64)).max() < 1e-10
    Pd = st.dense_Pinv_band(0.6)
    assert np.abs(Pd - Pd.T).max() < 1e-12 * np.abs(Pd).max()


def test_band_preconditioner_eigen_form_equals_direct_inverse():
    """Eq. PreconFFT_ECS via eigenvectors equals F^-1 (K~ - E)^-1 F computed
    by plain per-band solves (no eigen-decomposition)."""
    st = S.Stationary1D(_small(128))
    r = np.random.default_rng(5).standard_normal(128) + 0j
    a = st.precond_band(r, 1.1, use_eig=True)
    b = st.precond_band(r, 1.1, use_eig=False)
    assert np.abs(a - b).max() < 1e-11 * np.abs(b).max()


def test_band_matrix_is_galerkin_of_Ka():
    """K~ restricted to a band equals the Galerkin matrix of
    K_a = -1/2 d/dx q^-2 d/dx in the Fourier basis (Sec. III, the operator
    K_a): <phi_n|K_a|phi_m> = 1/2 k_n k_m <phi_n|q^-2|phi_m>, each computed by
    the grid quadrature directly."""
    p = _small(64)
    st = S.Stationary1D(p)
    L = p.b - p.a
    phi = lambda k: np.exp(1j * k * p.x) / np.sqrt(L)
    iq2 = p.q ** -2.0
    (m0, w) = st.bands[3]
    Kl = st.Kls[3]
    for u in range(w):
        for v in range(w):
            kn, km = p.k[m0 + u], p.k[m0 + v]
            # integrate (d phi_n)^* q^-2 (d phi_m)/2 by the grid rule
            val = 0.5 * np.sum(np.conj(1j * kn * phi(kn)) * iq2 * (1j * km * phi(km))) * p.h
            assert abs(val - Kl[u, v]) < 1e-12 * abs(Kl).max()


def test_preconditioners_exact_for_free_unscaled_problem():
    """q = 1 and U = 0: A = F^-1 (K - E) F, so the simple preconditioner is
    A^-1 exactly (Eq. PreconFFT) and PCG converges in one iteration; the
    banded one reduces to it because Q = I makes every K_l diagonal."""
    p = _small(64, theta=0.0, potential=False)
    st = S.Stationary1D(p)
    f = np.random.default_rng(9).standard_normal(64) + 0j
    E = 0.37
    for pc in (st.precond_simple, st.precond_band):
        x, it, hist = S.cocg(lambda v: st.apply_A(v, E), lambda r: pc(r, E), f, tol=1e-12)
        assert it == 1 and hist[-1] < 1e-12
    X, lam = st.dense_X()
    assert np.abs(np.sort_complex(lam) - np.sort_complex(st.K + 0j)).max() < 1e-12


@pytest.mark.parametrize("kind", [T.SHARP, T.SECS])
def test_cocg_matches_dense_lu_1d(kind):
    """COCG (Sec. III) converges to the dense LU solution of Eq. linsys."""
    p = _small(64, theta=0.5, kind=kind)
    st = S.Stationary1D(p)
    E = 0.9
    A = st.dense_A(E)
    f = np.exp(-(p.x - 2.0) ** 2) + 0j
    xs = np.linalg.solve(A, f)
    for pc in (st.precond_simple, st.precond_band):
        x, it, hist = S.cocg(lambda v: st.apply_A(v, E), lambda r: pc(r, E), f, tol=1e-10)
        assert hist[-1] < 1e-10
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
        assert np.linalg.norm(A @ x - f) / np.linalg.norm(f) < 1e-10


def test_cocg_matches_dense_lu_2d():
    """2D form (sum of 1D terms) against a dense LU solve on a 16 x 16 grid;
    the dense A is built from Kronecker products of the 1D pieces."""
    n = 16
    box = (-12.0, 12.0, -12.0, 12.0)
    p2 = P.Problem2D(n, n, box, R0=8.0, theta=0.4, a2=1.0)
    st = S.Stationary2D(p2, nbw=4, kind=T.SHARP, R0=8.0, theta=0.4)
    E = 0.6
    F = np.exp(1j * np.outer(p2.kx, p2.x)) / np.sqrt(n)
    K1 = 0.5 * p2.kx ** 2
    Kd = F.conj().T @ np.diag(K1) @ F
    Cx = T.dense_from_tridiag(*p2.Cx)
    Cy = T.dense_from_tridiag(*p2.Cy)
    I = np.eye(n)
    A = (np.kron(I, Kd + Cx) + np.kron(Kd + Cy, I) + np.diag(p2.U.ravel())
         - E * np.eye(n * n))
    v = np.random.default_rng(2).standard_normal((n, n)) + 0j
    assert np.abs((A @ v.ravel()).reshape(n, n) - st.apply_A(v, E)).max() < 1e-11
    f = np.exp(-(p2.x[None, :] ** 2 + p2.y[:, None] ** 2) / 4) + 0j
    xs = np.linalg.solve(A, f.ravel()).reshape(n, n)
    for pc in (st.precond_simple, st.precond_band):
        x, it, hist = S.cocg(lambda u: st.apply_A(u, E), lambda r: pc(r, E), f, tol=1e-10)
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8


def test_2d_band_preconditioner_is_kron_of_1d():
    """The 2D banded preconditioner equals the dense
    F^dag (X_x (x) X_y)^T (Lambda_x (+) Lambda_y - E)^-1 (X_x (x) X_y) F."""
    n = 16
    box = (-12.0, 12.0, -12.0, 12.0)
    p2 = P.Problem2D(n, n, box, R0=8.0, theta=0.4, a2=1.0)
    st = S.Stationary2D(p2, nbw=4, kind=T.SHARP, R0=8.0, theta=0.4)
    Fx = np.exp(1j * np.outer(p2.kx, p2.x)) / np.sqrt(n)
    Fy = np.exp(1j * np.outer(p2.ky, p2.y)) / np.sqrt(n)
    Xs = []
    for a in st.axes:
        X = np.zeros((n, n), dtype=complex)
        for (m0, w), (l, Xl) in zip(a["bands"], a["eig"]):
            X[m0:m0 + w, m0:m0 + w] = Xl
        Xs.append(X)
    lx, ly = st.lambdas()
    F2 = np.kron(Fy, Fx)
    X2 = np.kron(Xs[1], Xs[0])
    lam2 = (ly[:, None] + lx[None, :]).ravel()
    E = 0.45
    Pd = F2.conj().T @ X2.T @ np.diag(1 / (lam2 - E)) @ X2 @ F2
    r = np.random.default_rng(4).standard_normal((n, n)) + 0j
    assert np.abs((Pd @ r.ravel()).reshape(n, n) - st.precond_band(r, E)).max() < 1e-10 * np.abs(Pd).max()
