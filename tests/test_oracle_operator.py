"""Pins of the oracle's space discretisation and substep solves (not GPU).

Each test checks the FP64 oracle against something fixed outside it: the
closed-form eigen-pairs of the discrete Laplacian (Sec. 2.2 with the
stability function of eq. stab_func_FIE), the continuous operator of
eq. cont_problem (second-order consistency), a dense direct solve assembled
from the oracle's *operator* path (a different code path from its line
solves), symmetry, the maximum principle, and for the DD splitting the
partition-of-unity identities of Sec. 2.1.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import analysis as an
from paper_2502_08370_gb300 import workloads as wl


def dense_A(p, m):
    """Dense matrix of A_m built column by column from the oracle's apply_A."""
    n = p.size
    A = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        A[:, j] = orc.apply_A(p, m, e).reshape(-1)
    return A


@pytest.mark.parametrize("n", [(7, 5), (6, 4, 5)])
@pytest.mark.parametrize("c", [0.0, 3.0])
def test_sine_modes_are_eigenvectors(n, c):
    """Constant a: A_m sin-mode = (lambda_{p_m} - c/M) sin-mode, lambda_p = -(4/h^2) sin^2(p pi h/2)."""
    p = orc.Problem(n, c=c)
    M = len(n)
    rng = np.random.default_rng(0)
    for _ in range(4):
        ps = [int(rng.integers(1, nd + 1)) for nd in n]
        phi = an.sine_mode(ps, n)
        for m in range(M):
            lam = an.laplacian_eigenvalue(ps[m], n[m]) - c / M
            np.testing.assert_allclose(orc.apply_A(p, m, phi), lam * phi, rtol=0, atol=1e-9 * abs(lam))


@pytest.mark.parametrize("n", [(9, 6), (5, 6, 7)])
def test_fie_step_amplification_factor(n):
    """One FIE step on a sine mode multiplies it by R_FIE(tau lam_1, ..., tau lam_M) (eq. stab_func_FIE)."""
    p = orc.Problem(n)
    tau = 0.013
    rng = np.random.default_rng(1)
    for _ in range(5):
        ps = [int(rng.integers(1, nd + 1)) for nd in n]
        phi = an.sine_mode(ps, n)
        R = an.R_FIE(*[tau * an.laplacian_eigenvalue(ps[m], n[m]) for m in range(len(n))])
        np.testing.assert_allclose(orc.fie_step(p, tau, phi), R * phi, rtol=0, atol=1e-13)
        # and each substep separately: 1/(1 - tau lam_m)
        x = phi
        for m in range(len(n)):
            x = orc.substep_solve(p, m, tau, x)
            r = np.prod([1.0 / (1.0 - tau * an.laplacian_eigenvalue(ps[j], n[j])) for j in range(m + 1)])
            np.testing.assert_allclose(x, r * phi, rtol=0, atol=1e-13)


def test_variable_coefficient_consistency_second_order():
    """(A_0 u)(x) -> d/dx(a du/dx) at O(h^2) for smooth a, u (eq. cont_problem, Sec. 5)."""
    errs = []
    for n in (15, 31, 63):
        h = 1.0 / (n + 1)
        xb = np.arange(n + 2) * h
        x = xb[1:-1]
        y = x
        # a(x, y) = 2 + sin(x) cos(2y) on the nodal grid incl. boundary
        A = 2.0 + np.outer(np.cos(2 * xb), np.sin(xb))  # shape (y, x): a = 2 + sin(x) cos(2y)
        u = np.outer(np.sin(np.pi * y), np.sin(np.pi * x))  # zero on the boundary
        p = orc.Problem((n, n), a=A)
        got = orc.apply_A(p, 0, u)
        a_c = 2.0 + np.outer(np.cos(2 * y), np.sin(x))
        ax = np.outer(np.cos(2 * y), np.cos(x))
        ux = np.pi * np.outer(np.sin(np.pi * y), np.cos(np.pi * x))
        uxx = -np.pi ** 2 * u
        exact = ax * ux + a_c * uxx
        errs.append(np.max(np.abs(got - exact)))
        got_y = orc.apply_A(p, 1, u)
        ay = np.outer(-2 * np.sin(2 * y), np.sin(x))
        uy = np.pi * np.outer(np.cos(np.pi * y), np.sin(np.pi * x))
        exact_y = ay * uy + a_c * uxx
        assert np.max(np.abs(got_y - exact_y)) < 40 * h * h * 10
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.5 < r2 < 4.5, errs


@pytest.mark.parametrize("n", [(6, 5), (4, 5, 3)])
def test_substep_solve_matches_dense(n):
    """Line solves (Thomas) == dense solve of (I - tau A_m) from the operator path, random a."""
    rng = np.random.default_rng(2)
    a = np.exp(0.5 * rng.standard_normal([v + 2 for v in reversed(n)]))
    p = orc.Problem(n, a=a, c=0.7)
    tau = 0.05
    b = rng.standard_normal(p.size)
    for m in range(len(n)):
        A = dense_A(p, m)
        x_ref = np.linalg.solve(np.eye(p.size) - tau * A, b)
        x = orc.substep_solve(p, m, tau, b).reshape(-1)
        np.testing.assert_allclose(x, x_ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [(6, 7), (4, 3, 5)])
def test_operator_symmetric_and_negative(n):
    rng = np.random.default_rng(3)
    a = np.exp(0.5 * rng.standard_normal([v + 2 for v in reversed(n)]))
    p = orc.Problem(n, a=a, c=0.3)
    for m in range(len(n)):
        A = dense_A(p, m)
        np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-10 * np.abs(A).max())
        assert np.linalg.eigvalsh(A).max() < 0


def test_maximum_principle_every_substep():
    """f = 0: each (I - tau A_m)^{-1} is a nonnegative contraction in the max norm."""
    rng = np.random.default_rng(4)
    n = (12, 9, 7)
    a = np.exp(0.7 * rng.standard_normal([v + 2 for v in reversed(n)]))
    p = orc.Problem(n, a=a)
    u = rng.standard_normal(p.size)
    for m in range(3):
        v = orc.substep_solve(p, m, 0.2, u)
        assert np.abs(v).max() <= np.abs(u).max() * (1 + 1e-14)
        pos = orc.substep_solve(p, m, 0.2, np.abs(u))
        assert pos.min() >= 0.0
        u = v.reshape(-1)


# ---------------------------------------------------------------- DD splitting
def dd_problem(n=(31, 23), boxes=(4, 3), overlap_cells=3, a=None, c=0.0):
    return orc.Problem(n, a=a, c=c, split="dd", boxes=boxes, overlap=overlap_cells / (n[0] + 1.0))


def test_partition_of_unity():
    """sum_j rho_j = 1, 0 <= rho_j <= 1, rho_j = 1 in a core, 0 away from its boxes (Sec. 2.1)."""
    p = dd_problem()
    assert p.M == 4
    rng = np.random.default_rng(5)
    for x, y in rng.uniform(0, 1, (500, 2)):
        r = [orc.rho(p, j, x, y) for j in range(4)]
        assert abs(sum(r) - 1.0) < 1e-15
        assert min(r) >= 0.0 and max(r) <= 1.0
    # centre of box (1,1) belongs to colour (1%2)+2*(1%2) = 3 only
    bx, by = 1, 1
    xc, yc = (bx + 0.5) / 4, (by + 0.5) / 3
    assert orc.rho(p, 3, xc, yc) == 1.0
    # 1-D partition: telescoping sum and the cos^2 ramp's midpoint value 1/2
    w = 0.1
    for x in np.linspace(0, 1, 101):
        assert abs(sum(orc.phi1d(b, 5, w, x) for b in range(5)) - 1.0) < 1e-15
    assert abs(orc.phi1d(0, 5, w, 0.2) - 0.5) < 1e-15


def test_dd_operators_sum_to_dimensional_operator():
    """sum_j A_j^DD = A = sum_j A_j^dim (Sec. 2.1), variable a and reaction."""
    rng = np.random.default_rng(6)
    n = (21, 17)
    a = np.exp(0.4 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    pdd = dd_problem(n, boxes=(3, 2), overlap_cells=2, a=a, c=1.5)
    pdim = orc.Problem(n, a=a, c=1.5)
    for _ in range(3):
        u = rng.standard_normal(pdim.size)
        s_dd = sum(orc.apply_A(pdd, j, u) for j in range(pdd.M))
        s_dim = sum(orc.apply_A(pdim, j, u) for j in range(2))
        np.testing.assert_allclose(s_dd, s_dim, rtol=0, atol=1e-11 * np.abs(s_dim).max())


def test_dd_substep_matches_dense_and_is_block_diagonal():
    rng = np.random.default_rng(7)
    n = (13, 11)
    a = np.exp(0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    p = dd_problem(n, boxes=(3, 2), overlap_cells=2, a=a, c=0.5)
    tau = 0.03
    b = rng.standard_normal(p.size)
    for j in range(p.M):
        A = dense_A(p, j)
        np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-10 * np.abs(A).max())
        x_ref = np.linalg.solve(np.eye(p.size) - tau * A, b)
        x = orc.substep_solve(p, j, tau, b).reshape(-1)
        np.testing.assert_allclose(x, x_ref, rtol=1e-12, atol=1e-13)
        # no coupling between nodes of different boxes of the colour
        box_id = -np.ones(n[::-1], dtype=int)
        for by in range(2):
            for bx in range(3):
                if (bx % 2) + 2 * (by % 2) != j:
                    continue
                xr, yr = orc.box_range(p, 0, bx), orc.box_range(p, 1, by)
                box_id[yr[0] - 1:yr[1], xr[0] - 1:xr[1]] = by * 3 + bx
        bid = box_id.reshape(-1)
        r, c = np.nonzero(np.abs(A) > 0)
        off = r != c
        assert np.all(bid[r[off]] == bid[c[off]]) and np.all(bid[r[off]] >= 0)


def test_dd_config_geometry():
    """1023^2, 8x8 boxes, overlap 8 cells: interior boxes span 137 nodes, edge boxes 132."""
    cfg = wl.dd2d_1023(n=1023)
    p = orc.Problem(cfg["n"], split="dd", boxes=cfg["boxes"], overlap=cfg["overlap"])
    widths = [orc.box_range(p, 0, b) for b in range(8)]
    assert widths[0] == (1, 132) and widths[7] == (892, 1023)
    for b in range(1, 7):
        lo, hi = widths[b]
        assert (lo, hi) == (128 * b - 4, 128 * b + 132)


@pytest.mark.parametrize("n", [(9, 8), (6, 5, 7)])
def test_fie_steps_are_affine_increment_form(n):
    """The FIE step is affine in the state (eq. FIE_method: the source enters as a fixed
    right-hand-side term), so for any two states the difference of their propagations equals
    the source-free propagation of their difference.  This is the identity the FP32 coarse
    increment form uses: G(U^k) - G(U^{k-1}) = B (U^k - U^{k-1}).  A dropped or doubled source
    term, or a source scaled by the state, breaks it."""
    rng = np.random.default_rng(5)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    src_t = 1.0 + np.sin(np.arange(20) * 0.4)
    with_src = orc.Problem(n, a=a, c=0.3, src=src, src_t=src_t)
    no_src = orc.Problem(n, a=a, c=0.3)
    u, v = rng.standard_normal(n[::-1]), rng.standard_normal(n[::-1])
    tau, steps = 0.07, 3
    d = orc.propagate(with_src, tau, steps, u, t0=2) - orc.propagate(with_src, tau, steps, v, t0=2)
    b = orc.propagate(no_src, tau, steps, u - v, t0=2)
    assert np.abs(d - b).max() <= 1e-13 * np.abs(b).max()
    # and the source does contribute: the propagations themselves differ from the source-free ones
    assert np.abs(orc.propagate(with_src, tau, steps, u, t0=2) - orc.propagate(no_src, tau, steps, u, t0=2)).max() > 1e-3
