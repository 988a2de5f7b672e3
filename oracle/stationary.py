"""Oracle for the stationary ECS equation (Sec. III): the matrix A, the simple
FFT preconditioner (Eq. PreconFFT), the ECS-friendly banded preconditioner
(Eqs. Prec_eigen_eq, K_l, PreconFFT_ECS) and complex-symmetric conjugate
gradients, in plain FP64 numpy.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Conventions.  The paper's DFT matrix is F_{nj} = phi_n(x_j) sqrt(h) =
exp(i k_n x_j)/sqrt(N) (Sec. II, Eq. Fmatrix), unitary, F^{-1} = F^dagger.
Momenta k_n follow the FFT ordering of ``tables.kgrid``.  Small problems are
built as dense matrices from that definition; large ones apply the same
operators through numpy's FFT (a library primitive).
"""
from __future__ import annotations

import numpy as np

from . import tables as T

# ----------------------------------------------------------------- basis ---


def dft_matrix(x, k):
    """F_{nj} = exp(i k_n x_j)/sqrt(N) (Sec. II, Eq. Fmatrix)."""
    n = len(x)
    return np.exp(1j * np.outer(k, x)) / np.sqrt(n)


def to_k(r, x0, k):
    """F r via FFT: (F r)_n = e^{i k_n x_0} sum_j e^{2 pi i n j/N} r_j / sqrt(N)."""
    n = r.shape[-1]
    return np.exp(1j * k * x0) * np.fft.ifft(r, axis=-1) * np.sqrt(n)


def from_k(c, x0, k):
    """F^dagger c via FFT."""
    n = c.shape[-1]
    return np.fft.fft(np.exp(-1j * k * x0) * c, axis=-1) / np.sqrt(n)


# ------------------------------------------------------------ band split ---


def band_split(n: int, nbw: int = 10):
    """Spectrum split of Sec. III (paragraph after Fig. 1): singleton bands
    {k_1 = 0} and {k_{N/2+1}} (Nyquist); bands of constant width N_BW; the two
    bands next to the Nyquist index (one on each sign of k, mirror images)
    take the remaining modes, N_BW <= N_l <= 2 N_BW - 1.

    Returns a list of (first index, width) in 0-based FFT ordering."""
    if n < 4:
        return [(m, 1) for m in range(n)]
    half = n // 2
    npos = half - 1                       # m = 1 .. N/2-1 (k > 0)
    q, r = divmod(npos, nbw)
    widths = [npos] if q == 0 else [nbw] * (q - 1) + [nbw + r]
    bands = [(0, 1)]
    m = 1
    for w in widths:                      # positive side, away from k = 0
        bands.append((m, w))
        m += w
    bands.append((half, 1))               # Nyquist singleton
    for w in reversed(widths):            # negative side: mirror images
        bands.append((m + 1, w))          # m + 1 = first index after Nyquist
        m += w
    return bands


def q_fourier(x, q, L, dmax):
    """g(d) = (1/N) sum_j exp(2 pi i d x_j / L) q(x_j)^{-2}, |d| <= dmax: the
    overlap Q_{nm} = <phi_n| q^{-2} |phi_m> = g(m - n) of Sec. III (the
    integral under Eq. K_l taken by the grid's own quadrature, a reading)."""
    n = len(x)
    iq2 = np.zeros(n, dtype=np.complex128)
    fin = np.isfinite(q)
    iq2[fin] = q[fin] ** -2.0
    d = np.arange(-dmax, dmax + 1)
    g = np.exp(2j * np.pi * np.outer(d, x) / L) @ iq2 / n
    return {int(dd): g[i] for i, dd in enumerate(d)}


def band_matrices(k, g, bands):
    """K_l with [K_l]_{uv} = 1/2 k_u k_v g(v - u) on each band (Eq. K_l)."""
    out = []
    for (m0, w) in bands:
        idx = np.arange(m0, m0 + w)
        kk = k[idx]
        G = np.array([[g[int(v - u)] for v in idx] for u in idx])
        out.append(0.5 * np.outer(kk, kk) * G)
    return out


def band_eig(Kls):
    """Eigen-decomposition of every K_l (Eq. Prec_eigen_eq): returns per band
    (lambda, X_l) with the rows of X_l the eigenvectors chi_nu, normalised by
    the unconjugated chi^T chi = 1 so that X_l^{-1} = X_l^T (Sec. III)."""
    out = []
    for K in Kls:
        lam, V = np.linalg.eig(K)
        nrm = np.sqrt(np.sum(V * V, axis=0))
        V = V / nrm
        out.append((lam, V.T.copy()))
    return out


class Stationary1D:
    """A = F^-1 K F + C + U - E I (Sec. III, the matrix under Eq. linsys)."""

    def __init__(self, prob, nbw=10):
        self.p = prob
        self.n = prob.n
        self.x0 = prob.x[0]
        self.L = prob.b - prob.a
        self.K = 0.5 * prob.k ** 2
        self.bands = band_split(self.n, nbw)
        wmax = max(w for _, w in self.bands)
        self.g = q_fourier(prob.x, prob.q, self.L, wmax)
        self.Kls = band_matrices(prob.k, self.g, self.bands)
        self.eig = band_eig(self.Kls)

    # ---- operators applied through the FFT
    def apply_A(self, psi, E):
        p = self.p
        kin = np.fft.ifft(self.K * np.fft.fft(psi))
        cps = p.Cs * np.roll(psi, 1) + p.Cd * psi + p.Cu * np.roll(psi, -1)
        return kin + cps + (p.U0 - E) * psi

    def precond_simple(self, r, E):
        """P^-1 = F^-1 (K - E)^-1 F (Eq. PreconFFT)."""
        return np.fft.ifft(np.fft.fft(r) / (self.K - E))

    def precond_band(self, r, E, use_eig=True):
        """P^-1 = F^-1 X^-1 (Lambda - E)^-1 X F (Eq. PreconFFT_ECS); with
        use_eig=False the same operator F^-1 (K~ - E)^-1 F by direct per-band
        solves (no eigen-decomposition)."""
        c = to_k(r, self.x0, self.p.k)
        out = np.zeros_like(c)
        for (m0, w), Kl, (lam, X) in zip(self.bands, self.Kls, self.eig):
            seg = c[m0:m0 + w]
            if use_eig:
                out[m0:m0 + w] = X.T @ ((X @ seg) / (lam - E))
            else:
                out[m0:m0 + w] = np.linalg.solve(Kl - E * np.eye(w), seg)
        return from_k(out, self.x0, self.p.k)

    # ---- dense forms (tiny N only)
    def dense_F(self):
        return dft_matrix(self.p.x, self.p.k)

    def dense_A(self, E):
        p = self.p
        F = self.dense_F()
        A = F.conj().T @ np.diag(self.K) @ F
        A = A + T.dense_from_tridiag(p.Cs, p.Cd, p.Cu) + np.diag(p.U0) - E * np.eye(self.n)
        return A

    def dense_Ktilde(self):
        Kt = np.zeros((self.n, self.n), dtype=np.complex128)
        for (m0, w), Kl in zip(self.bands, self.Kls):
            Kt[m0:m0 + w, m0:m0 + w] = Kl
        return Kt

    def dense_X(self):
        X = np.zeros((self.n, self.n), dtype=np.complex128)
        lam = np.zeros(self.n, dtype=np.complex128)
        for (m0, w), (l, Xl) in zip(self.bands, self.eig):
            X[m0:m0 + w, m0:m0 + w] = Xl
            lam[m0:m0 + w] = l
        return X, lam

    def dense_Pinv_band(self, E):
        F = self.dense_F()
        X, lam = self.dense_X()
        return F.conj().T @ X.T @ np.diag(1.0 / (lam - E)) @ X @ F


class Stationary2D:
    """2D form: A = F^-1 (Kx + Ky) F + C_x (x) I + I (x) C_y + U - E, psi
    stored [ny][nx].  The banded preconditioner uses X = X_x (x) X_y and
    Lambda = lambda_x + lambda_y (a reading of Sec. III's remark that the FFT
    preconditioner generalises directly to several dimensions: K_a is a sum
    of one-dimensional terms)."""

    def __init__(self, prob, nbw=10, kind=T.SHARP, R0=None, theta=None, alpha=0.5):
        self.p = prob
        ax, bx, ay, by = prob.box
        self.K = 0.5 * (prob.kx[None, :] ** 2 + prob.ky[:, None] ** 2)
        self.axes = []
        for (n, a, b, xs, ks) in ((prob.nx, ax, bx, prob.x, prob.kx),
                                  (prob.ny, ay, by, prob.y, prob.ky)):
            q = T.q_contour(xs, kind, R0, b, theta, alpha)
            bands = band_split(n, nbw)
            wmax = max(w for _, w in bands)
            g = q_fourier(xs, q, b - a, wmax)
            Kls = band_matrices(ks, g, bands)
            self.axes.append(dict(x0=xs[0], k=ks, bands=bands, Kls=Kls, eig=band_eig(Kls)))

    def apply_A(self, psi, E):
        p = self.p
        kin = np.fft.ifft2(self.K * np.fft.fft2(psi))
        cxs, cxd, cxu = p.Cx
        cys, cyd, cyu = p.Cy
        cx = cxs[None, :] * np.roll(psi, 1, axis=1) + cxd[None, :] * psi + cxu[None, :] * np.roll(psi, -1, axis=1)
        cy = cys[:, None] * np.roll(psi, 1, axis=0) + cyd[:, None] * psi + cyu[:, None] * np.roll(psi, -1, axis=0)
        return kin + cx + cy + (p.U - E) * psi

    def precond_simple(self, r, E):
        return np.fft.ifft2(np.fft.fft2(r) / (self.K - E))

    def _axis_apply(self, c, ax_i, op):
        a = self.axes[ax_i]
        out = np.zeros_like(c)
        for (m0, w), (lam, X) in zip(a["bands"], a["eig"]):
            M = X if op == "X" else X.T
            if ax_i == 0:   # along x (last axis)
                out[:, m0:m0 + w] = c[:, m0:m0 + w] @ M.T
            else:           # along y (first axis)
                out[m0:m0 + w, :] = M @ c[m0:m0 + w, :]
        return out

    def lambdas(self):
        res = []
        for a in self.axes:
            lam = np.zeros(len(a["k"]), dtype=np.complex128)
            for (m0, w), (l, _) in zip(a["bands"], a["eig"]):
                lam[m0:m0 + w] = l
            res.append(lam)
        return res

    def precond_band(self, r, E):
        ax, ay = self.axes
        c = to_k(r, ax["x0"], ax["k"])                               # along x
        c = np.swapaxes(to_k(np.swapaxes(c, 0, 1), ay["x0"], ay["k"]), 0, 1)  # along y
        c = self._axis_apply(self._axis_apply(c, 0, "X"), 1, "X")
        lx, ly = self.lambdas()
        c = c / (lx[None, :] + ly[:, None] - E)
        c = self._axis_apply(self._axis_apply(c, 0, "XT"), 1, "XT")
        c = from_k(c, ax["x0"], ax["k"])
        c = np.swapaxes(from_k(np.swapaxes(c, 0, 1), ay["x0"], ay["k"]), 0, 1)
        return c


def cocg(apply_A, precond, f, tol=1e-8, maxit=1000):
    """Preconditioned conjugate gradients for complex-symmetric A (Sec. III,
    the paragraph after Eq. linsys): the unconjugated bilinear form r^T z
    replaces the inner product.  Stops when ||r||_2/||f||_2 < tol (Hermitian
    norms).  Returns (x, iterations, relative residual history)."""
    x = np.zeros_like(f)
    r = f.copy()
    fn = np.linalg.norm(f)
    z = precond(r)
    p = z.copy()
    rho = np.sum(r * z)
    hist = [np.linalg.norm(r) / fn]
    it = 0
    while hist[-1] >= tol and it < maxit:
        w = apply_A(p)
        alpha = rho / np.sum(p * w)
        x = x + alpha * p
        r = r - alpha * w
        it += 1
        hist.append(np.linalg.norm(r) / fn)
        if hist[-1] < tol:
            break
        z = precond(r)
        rho_new = np.sum(r * z)
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    return x, it, hist
