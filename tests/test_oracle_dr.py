"""Pins of the oracle's Douglas-Rachford step (eq. DR_method) and the Parareal/FIE-DR pairing
(Sec. 4.2), the next method on the path (not GPU).

- One DR step on a discrete sine mode multiplies it by R_DR(tau lam_1, ..., tau lam_M)
  (eq. stab_func_DR).
- The DR step equals its definition evaluated with dense matrices (variable a, reaction,
  source; dimensional and DD splittings).
- Splitting error: against the unsplit implicit Euler step, DR is third-order locally (its
  splitting error is second order, Sec. 2.2), FIE second-order.  A dropped -tau A_j U_n
  term or a wrong sign in the stage U_{n,0} changes these orders.
- Parareal/FIE-DR on a constant-coefficient problem equals the per-mode scalar recursion
  with G = R_FIE(z), F = R_DR(z/s)^s at every iteration; finite termination is bitwise.
- Theorem 2 and its corollary: K_FIE-DR(z, s) < 1 on (-inf, 0)^M, approaching 1 for large |z|.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import analysis as an


def dense_ops(p, n):
    """A_m as dense matrices, column by column from the oracle's operator application."""
    size = int(np.prod(n))
    mats = []
    e = np.zeros(size)
    for m in range(p.M):
        A = np.zeros((size, size))
        for j in range(size):
            e[:] = 0.0
            e[j] = 1.0
            A[:, j] = orc.apply_A(p, m, e.reshape(n[::-1])).reshape(-1)
        mats.append(A)
    return mats


@pytest.mark.parametrize("n", [(9, 6), (5, 6, 7)])
@pytest.mark.parametrize("tau", [0.013, 0.4])
def test_dr_step_amplification_factor(n, tau):
    p = orc.Problem(n)
    rng = np.random.default_rng(2)
    for _ in range(5):
        ps = [int(rng.integers(1, nd + 1)) for nd in n]
        phi = an.sine_mode(ps, n)
        z = [tau * an.laplacian_eigenvalue(ps[m], n[m]) for m in range(len(n))]
        R = an.R_DR(*z)
        np.testing.assert_allclose(orc.dr_step(p, tau, phi), R * phi, rtol=0, atol=1e-13 * max(1.0, abs(R)))


@pytest.mark.parametrize("case", ["dim2", "dim3", "dd", "dd_tensor"])
def test_dr_step_matches_dense_definition(case):
    rng = np.random.default_rng(3)
    if case == "dim2":
        n, kw = (6, 5), {}
    elif case == "dim3":
        n, kw = (4, 3, 5), {}
    elif case == "dd":
        n, kw = (9, 8), dict(split="dd", boxes=(2, 2), overlap=2.0 / 10)
    else:  # full tensor (Sec. 5.2) with a second separable source term
        n = (9, 8)
        kw = dict(split="dd", boxes=(2, 2), overlap=2.0 / 10, d12=0.2 + 0.05 * rng.standard_normal((10, 11)),
                  src2=rng.standard_normal((8, 9)), src2_t=np.cos(np.arange(10) * 0.3))
    a = np.exp(0.4 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    src_t = 1.0 + np.sin(np.arange(10) * 0.5)
    p = orc.Problem(n, a=a, c=0.7, src=src, src_t=src_t, **kw)
    u = rng.standard_normal(n[::-1])
    tau, t_end = 0.05, 3
    mats = dense_ops(p, n)
    I = np.eye(u.size)
    uf = u.reshape(-1)
    v = uf + tau * sum(A @ uf for A in mats) + tau * src.reshape(-1) * src_t[t_end]
    if "src2" in kw:
        v = v + tau * kw["src2"].reshape(-1) * kw["src2_t"][t_end]
    for A in mats:
        v = np.linalg.solve(I - tau * A, v - tau * A @ uf)
    got = orc.dr_step(p, tau, u, t_end=t_end).reshape(-1)
    assert np.abs(got - v).max() <= 1e-12 * np.abs(v).max()


def test_splitting_error_orders_against_implicit_euler():
    """Local error of one step against the unsplit implicit Euler step (I - tau A)^{-1} u on a
    smooth state, variable coefficient (non-commuting A_x, A_y): halving tau divides the FIE
    error by ~4 (second order) and the DR error by ~8 (third order)."""
    n = (11, 9)
    xs = np.arange(1, n[0] + 1) / (n[0] + 1.0)
    ys = np.arange(1, n[1] + 1) / (n[1] + 1.0)
    X = np.add.outer(0 * ys, xs)
    Y = np.add.outer(ys, 0 * xs)
    a_x = np.arange(0, n[0] + 2) / (n[0] + 1.0)
    a_y = np.arange(0, n[1] + 2) / (n[1] + 1.0)
    a = 1.0 + 0.5 * np.outer(np.sin(np.pi * a_y), np.cos(2 * np.pi * a_x))
    p = orc.Problem(n, a=a)
    u = np.sin(np.pi * X) * np.sin(np.pi * Y) + 0.3 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y)
    A = sum(dense_ops(p, n))
    I = np.eye(u.size)
    errs = {"fie": [], "dr": []}
    taus = [2e-4, 1e-4, 5e-5]
    for tau in taus:
        be = np.linalg.solve(I - tau * A, u.reshape(-1))
        errs["fie"].append(np.abs(orc.fie_step(p, tau, u).reshape(-1) - be).max())
        errs["dr"].append(np.abs(orc.dr_step(p, tau, u).reshape(-1) - be).max())
    r_fie = [errs["fie"][i] / errs["fie"][i + 1] for i in range(2)]
    r_dr = [errs["dr"][i] / errs["dr"][i + 1] for i in range(2)]
    assert all(3.5 < r < 4.5 for r in r_fie), r_fie
    assert all(6.5 < r < 9.0 for r in r_dr), r_dr
    assert errs["dr"][-1] < 0.1 * errs["fie"][-1]


def test_parareal_fie_dr_equals_modal_recursion_every_iteration():
    n = (15, 11)
    T, N, s = 1.0, 6, 8
    rng = np.random.default_rng(20)
    modes = [(1, 1)] + [(int(rng.integers(1, n[0] + 1)), int(rng.integers(1, n[1] + 1))) for _ in range(5)]
    amps = np.array([1.0] + list(rng.uniform(-1, 1, 5)))
    phis = [an.sine_mode(m, n) for m in modes]
    u0 = sum(A * ph for A, ph in zip(amps, phis))
    p = orc.Problem(n)
    lx = np.array([an.laplacian_eigenvalue(m[0], n[0]) for m in modes])
    ly = np.array([an.laplacian_eigenvalue(m[1], n[1]) for m in modes])
    DT = T / N
    rg = an.R_FIE(lx * DT, ly * DT)
    rf = an.R_DR(lx * DT / s, ly * DT / s) ** s
    Y = np.array([amps * rg ** j for j in range(N + 1)])  # k = 0: the coarse sweep
    for k in range(0, N + 1):
        if k == 0:
            U = orc.coarse_sequential(p, T, N, 1, s, u0)
        else:
            U, _, it = orc.parareal(p, T, N, 1, s, u0, tol=0.0, max_iter=k, fine="dr")
            assert it == k
        for j in range(N + 1):
            ref = sum(Y[j, i] * phis[i] for i in range(len(modes)))
            np.testing.assert_allclose(U[j], ref, rtol=0, atol=1e-13)
        Y = an.scalar_parareal_iterate(Y, rg, rf)


@pytest.mark.parametrize("split", ["dim", "dd"])
def test_parareal_fie_dr_finite_termination_bitwise(split):
    rng = np.random.default_rng(21)
    n = (12, 10)
    a = np.exp(0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    N, s, T = 5, 4, 0.3
    src = rng.standard_normal(n[::-1])
    src_t = np.cos(np.arange(N * s + 1) * 0.2)
    kw = dict(split="dd", boxes=(3, 2), overlap=2.0 / (n[0] + 1)) if split == "dd" else {}
    p = orc.Problem(n, a=a, c=0.1, src=src, src_t=src_t, **kw)
    u0 = rng.standard_normal(n[::-1])
    fine = orc.fine_sequential_dr(p, T, N, s, u0)
    for k in (1, 3, N):
        U, _, it = orc.parareal(p, T, N, 1, s, u0, tol=0.0, max_iter=k, fine="dr")
        assert it == k
        for j in range(k + 1):
            assert np.array_equal(U[j], fine[j]), (k, j)


def test_theorem2_convergence_factor_below_one():
    """K_FIE-DR(z, s) < 1 on (-inf, 0)^M for s >= 1 (Theorem 2 and its corollary).  Unlike
    FIE-FIE (<= 1/3), the factor approaches 1 for large |z| (DR is not L-stable)."""
    zs = -np.logspace(-3, 4, 40)
    for s in (1, 2, 5, 20, 100):
        for M in (2, 3):
            grids = np.meshgrid(*([zs] * M), indexing="ij")
            K = an.conv_factor([g.ravel() for g in grids], s, RF=an.R_DR, RG=an.R_FIE)
            assert np.all(K < 1.0), (s, M, K.max())
    K_big = an.conv_factor([np.array([-1e4]), np.array([-1e4])], 1, RF=an.R_DR, RG=an.R_FIE)
    assert K_big[0] > 0.9
