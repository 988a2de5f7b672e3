"""Oracle observables (TEST INFRASTRUCTURE, see ``oracle/__init__``).

The norm inside the unscaled region and the probability flux through its
edges at x = +-R0 are the two quantities the paper's t-SURFF analysis draws
from the propagated wave function (Sec. I and Sec. IV: the flux through the
boundary of the scaling region).  Both use samples psi_i = psi(x_i)."""
from __future__ import annotations

import numpy as np


def norm_inside(psi, x, h, R0):
    """h * sum_{|x_i| < R0} |psi_i|^2 (the paper's DVR norm, Sec. II, with the
    sqrt(h) factor of psi_i = sqrt(h) psi(x_i) written out)."""
    m = np.abs(x) < R0
    return float(h * np.sum(np.abs(psi[m]) ** 2))


def flux_at_edges(psi, x, h, R0):
    """j = Im(psi^* dpsi/dx) at x = -R0 and x = +R0.  R0 lies half-way between
    two grid points; psi there is the two-point mean and dpsi/dx the two-point
    difference (a reading: the paper gives no discretisation of the flux)."""
    out = []
    for edge in (-R0, R0):
        i = int(np.searchsorted(x, edge)) - 1          # x[i] < edge < x[i+1]
        pm = 0.5 * (psi[i] + psi[i + 1])
        dp = (psi[i + 1] - psi[i]) / h
        out.append(float(np.imag(np.conj(pm) * dp)))
    return out
