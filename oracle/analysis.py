"""Closed forms of the paper's analysis (arXiv 2502.08370, Sec. 2.2-4).

TEST INFRASTRUCTURE ONLY (part of the oracle).  Used as pins: the stability
functions, the convergence factor and the exact per-mode parareal recursion
for simultaneously diagonalisable splittings.
"""
from __future__ import annotations

import numpy as np


def R_FIE(*z):
    """Stability function of the FIE step (eq. stab_func_FIE): prod_j 1/(1 - z_j)."""
    r = 1.0
    for zj in z:
        r = r / (1.0 - np.asarray(zj))
    return r


def R_DR(*z):
    """Stability function of the Douglas-Rachford step (eq. stab_func_DR)."""
    return 1.0 + R_FIE(*z) * sum(np.asarray(zj) for zj in z)


def conv_factor(z, s, RF=R_FIE, RG=R_FIE):
    """Convergence factor K(z_1..z_M, s) of eq. conv_factor."""
    z = [np.asarray(zj) for zj in z]
    rg = RG(*z)
    rf = RF(*[zj / s for zj in z]) ** s
    return np.abs(rf - rg) / (1.0 - np.abs(rg))


def laplacian_eigenvalue(p, n):
    """Eigenvalue of the 1-D second-difference operator with Dirichlet ends on n
    interior nodes (h = 1/(n+1)) for the sine mode sin(p pi x_i): -(4/h^2) sin^2(p pi h / 2)."""
    h = 1.0 / (n + 1)
    return -(4.0 / h ** 2) * np.sin(p * np.pi * h / 2.0) ** 2


def sine_mode(ps, n):
    """Discrete sine mode prod_d sin(p_d pi x_d) on the interior grid, numpy shape (z,y,x)."""
    axes = []
    for p, nd in zip(ps, n):
        x = np.arange(1, nd + 1) / (nd + 1.0)
        axes.append(np.sin(p * np.pi * x))
    out = axes[0]
    for ax in axes[1:]:
        out = np.multiply.outer(ax, out)
    return out


def scalar_parareal(lams, T, N, s, y0, tol, max_iter=None):
    """Parareal/FIE-FIE on the partitioned Dahlquist problem y' = (sum lams) y
    (eq. part_Dahlquist) for many independent modes at once.

    lams: list of M arrays (one per splitting term, same shape = modes).
    Implements the recursion of Sec. 3 with G = R_FIE(lam*DT) and
    F = R_FIE(lam*DT/s)^s.  Returns (Y[n, mode] at the final k, per-k max increment
    over n>=1 of max |.| -- a function 'weight' may be applied by the caller)."""
    DT = T / N
    rg = R_FIE(*[l * DT for l in lams])
    rf = R_FIE(*[l * DT / s for l in lams]) ** s
    Y = [np.asarray(y0, dtype=float)]
    for n in range(N):
        Y.append(rg * Y[-1])
    Y = np.array(Y)
    return Y, rg, rf


def scalar_parareal_iterate(Y, rg, rf):
    """One parareal iteration on the modal amplitudes: new[n+1] = rg new[n] + rf Y[n] - rg Y[n]."""
    new = np.empty_like(Y)
    new[0] = Y[0]
    for n in range(Y.shape[0] - 1):
        new[n + 1] = rf * Y[n] + (rg * new[n] - rg * Y[n])
    return new
