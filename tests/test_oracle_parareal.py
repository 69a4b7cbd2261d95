"""Pins of the oracle's time integration and parareal iteration (not GPU).

- The whole parareal iteration on a constant-coefficient problem equals the
  scalar recursion of Sec. 3 applied mode by mode with the closed-form
  stability functions (eq. stab_func_FIE, Remark after eq. conv_factor).
- Finite termination (Sec. 3): U_n^k equals the sequential fine solution for
  n <= k, and after N iterations everywhere.
- Theorem 1 / Corollary (Sec. 4.1): K_FIE-FIE <= 1/3 on (-inf, 0)^M.
- First-order convergence in time and second order in space of the fine
  propagator against the manufactured solution of Sec. 5.
- The discrete adjoint: dot-product identity, dense Jacobian, finite differences.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import analysis as an
from paper_2502_08370_gb300 import workloads as wl


def modal_problem(n, modes, amps):
    u0 = np.zeros(n[::-1])
    for (p, q), A in zip(modes, amps):
        u0 += A * an.sine_mode((p, q), n)
    return u0


def test_parareal_equals_modal_recursion_every_iteration():
    n = (15, 11)
    T, N, s = 1.0, 6, 8
    rng = np.random.default_rng(10)
    modes = [(1, 1)] + [(int(rng.integers(1, n[0] + 1)), int(rng.integers(1, n[1] + 1))) for _ in range(5)]
    amps = [1.0] + list(rng.uniform(-1, 1, 5))
    u0 = modal_problem(n, modes, amps)
    p = orc.Problem(n)
    lx = np.array([an.laplacian_eigenvalue(m[0], n[0]) for m in modes])
    ly = np.array([an.laplacian_eigenvalue(m[1], n[1]) for m in modes])
    Y, rg, rf = an.scalar_parareal([lx, ly], T, N, s, np.array(amps), 0.0)
    phis = [an.sine_mode(m, n) for m in modes]
    for k in range(0, N + 1):
        if k == 0:
            U = orc.coarse_sequential(p, T, N, 1, s, u0)
        else:
            U, hist, it = orc.parareal(p, T, N, 1, s, u0, tol=0.0, max_iter=k)
            assert it == k
        for nn in range(N + 1):
            ref = sum(Y[nn, i] * phis[i] for i in range(len(modes)))
            np.testing.assert_allclose(U[nn], ref, rtol=0, atol=1e-13)
        Y = an.scalar_parareal_iterate(Y, rg, rf)


def test_parareal_iteration_count_heat2d_small():
    """Stopping rule: first k with max increment < tol; the count equals the modal prediction."""
    cfg = wl.heat2d_63(n=15, N=16, s=64)
    n = cfg["n"]
    amps, ps, qs = cfg["modes"]
    modes = [(1, 1)] + list(zip(ps, qs))
    A = [1.0] + list(amps)
    p = orc.Problem(n)
    U, hist, it = orc.parareal(p, cfg["T"], cfg["N"], 1, cfg["s"], cfg["u0"], cfg["tol"])
    lx = np.array([an.laplacian_eigenvalue(m[0], n[0]) for m in modes])
    ly = np.array([an.laplacian_eigenvalue(m[1], n[1]) for m in modes])
    Y, rg, rf = an.scalar_parareal([lx, ly], cfg["T"], cfg["N"], cfg["s"], np.array(A), 0.0)
    phis = np.array([an.sine_mode(m, n) for m in modes])
    k_pred = None
    for k in range(1, cfg["N"] + 1):
        Yn = an.scalar_parareal_iterate(Y, rg, rf)
        inc = max(np.abs(np.tensordot(Yn[j] - Y[j], phis, axes=1)).max() for j in range(1, cfg["N"] + 1))
        np.testing.assert_allclose(hist[k - 1], inc, rtol=1e-9, atol=1e-15)
        Y = Yn
        if inc < cfg["tol"]:
            k_pred = k
            break
    assert k_pred == it and it < cfg["N"]


@pytest.mark.parametrize("split", ["dim", "dd"])
def test_finite_termination_bitwise(split):
    """U_n^k == sequential fine solution for n <= k; k = N reproduces it everywhere (Sec. 3)."""
    rng = np.random.default_rng(11)
    n = (13, 10)
    a = np.exp(0.4 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    N, s, T = 5, 6, 0.3
    src = rng.standard_normal(n[::-1])
    src_t = np.cos(np.arange(N * s + 1) * 0.1)
    kw = dict(split="dd", boxes=(3, 2), overlap=2.0 / (n[0] + 1)) if split == "dd" else {}
    p = orc.Problem(n, a=a, c=0.2, src=src, src_t=src_t, **kw)
    u0 = rng.standard_normal(n[::-1])
    fine = orc.fine_sequential(p, T, N, s, u0)
    for k in range(1, N + 1):
        U, _, it = orc.parareal(p, T, N, 1, s, u0, tol=0.0, max_iter=k)
        assert it == k
        for j in range(k + 1):
            assert np.array_equal(U[j], fine[j]), (k, j)
    assert np.array_equal(U, fine)


def test_coarse_substeps_and_3d():
    """G with g > 1 substeps and 3-D dimensional splitting still terminate at the fine solution."""
    rng = np.random.default_rng(12)
    n = (5, 6, 4)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    p = orc.Problem(n, a=a, src=rng.standard_normal(n[::-1]))
    u0 = rng.standard_normal(n[::-1])
    N, s = 4, 6
    fine = orc.fine_sequential(p, 1.0, N, s, u0)
    U, hist, it = orc.parareal(p, 1.0, N, 2, s, u0, tol=0.0)
    assert it == N and np.array_equal(U, fine)


def test_convergence_factor_bound_theorem1():
    """K_FIE-FIE(z, s) <= 1/3 for z in (-inf,0)^M, M = 2, 3 (Theorem 1 and its Corollary)."""
    zs = -np.concatenate([np.logspace(-4, 6, 60)])
    for s in (1, 2, 20, 64, 1000):
        Z1, Z2 = np.meshgrid(zs, zs)
        K = an.conv_factor([Z1, Z2], s)
        assert K.max() <= 1.0 / 3.0
        if s >= 20:
            assert K.max() > 0.1  # a nontrivial factor, close to the plotted maximum
        if s == 1:
            assert K.max() == 0.0  # F = G when s = 1
        z3 = zs[::3]
        A, B, Cc = np.meshgrid(z3, z3, z3)
        assert an.conv_factor([A, B, Cc], s).max() <= 1.0 / 3.0
    # the proof's auxiliary inequality H(z1, z2) >= 4 on [-3, 0]^2 with equality at 0
    g = np.linspace(-3, 0, 121)
    Z1, Z2 = np.meshgrid(g, g)
    H = (1 - Z1) * (1 - Z2) * (3 * np.exp(Z1 + Z2) + 1)
    assert H.min() >= 4 - 1e-12 and abs(H[-1, -1] - 4) < 1e-12
    assert abs(H.max() - 16 * (1 + 3 / np.e ** 6)) < 1e-9


def test_observed_contraction_below_one_third():
    """Dimensional splitting, variable a: errors against the fine solution contract by <= 1/3 + slack."""
    rng = np.random.default_rng(13)
    n = (15, 15)
    a = np.exp(0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    p = orc.Problem(n, a=a)
    u0 = rng.standard_normal(n[::-1])
    N, s, T = 8, 10, 1.0
    fine = orc.fine_sequential(p, T, N, s, u0)
    prev = None
    for k in range(1, 5):
        U, _, _ = orc.parareal(p, T, N, 1, s, u0, tol=0.0, max_iter=k)
        err = np.abs(U - fine).max()
        if prev is not None and prev > 1e-13:
            assert err <= prev * (1.0 / 3.0 + 0.1)
        prev = err


def test_manufactured_solution_orders():
    """Fine solution vs u = sin(2 pi t) sin(2 pi x) sin(2 pi y) (Sec. 5): O(dt) and O(h^2)."""
    T = 1.0

    def err(n, N, s):
        S, st, exact = wl.manufactured((n, n), T, N, s)
        p = orc.Problem((n, n), src=S, src_t=st)
        U = orc.fine_sequential(p, T, N, s, np.zeros((n, n)))
        h = 1.0 / (n + 1)
        return max(np.sqrt(h * h * np.sum((U[j] - exact(j * T / N)) ** 2)) for j in range(1, N + 1))

    e_t = [err(31, 8, s) for s in (8, 16, 32)]
    assert 1.7 < e_t[0] / e_t[1] < 2.3 and 1.8 < e_t[1] / e_t[2] < 2.2, e_t
    # refine h by 2 and dt by 4 together: the error of an O(dt + h^2) scheme drops by 4
    e_h = [err(15, 8, 16), err(31, 8, 64), err(63, 8, 256)]
    assert 3.2 < e_h[0] / e_h[1] < 4.5 and 3.6 < e_h[1] / e_h[2] < 4.3, e_h


# ---------------------------------------------------------------- adjoint
def test_adjoint_matches_dense_jacobian():
    """dJ/du0 = Phi^T (U_N - target) where Phi is the dense propagator of all fine steps."""
    rng = np.random.default_rng(14)
    n = (4, 3)
    a = np.exp(0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    p = orc.Problem(n, a=a, c=0.4)
    N, s, T = 2, 3, 0.2
    u0 = rng.standard_normal(n[::-1])
    tgt = rng.standard_normal(n[::-1])
    nt = p.size
    Phi = np.empty((nt, nt))
    for j in range(nt):
        e = np.zeros(nt)
        e[j] = 1
        Phi[:, j] = orc.fine_sequential(p, T, N, s, e.reshape(n[::-1]))[-1].reshape(-1)
    J, gu, ga = orc.adjoint(p, T, N, s, u0, tgt)
    UN = Phi @ u0.reshape(-1)
    np.testing.assert_allclose(J, 0.5 * np.sum((UN - tgt.reshape(-1)) ** 2), rtol=1e-13)
    np.testing.assert_allclose(gu.reshape(-1), Phi.T @ (UN - tgt.reshape(-1)), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_finite_differences(dim):
    rng = np.random.default_rng(15 + dim)
    n = (6, 5) if dim == 2 else (4, 3, 5)
    shape_a = tuple(v + 2 for v in reversed(n))
    a = np.exp(0.3 * rng.standard_normal(shape_a))
    src = rng.standard_normal(n[::-1])
    N, s, T = 3, 4, 0.1
    src_t = 1.0 + 0.5 * np.sin(np.arange(N * s + 1))
    u0 = rng.standard_normal(n[::-1])
    tgt = rng.standard_normal(n[::-1])

    def J_of(aa, uu):
        pp = orc.Problem(n, a=aa, c=0.3, src=src, src_t=src_t)
        UN = orc.fine_sequential(pp, T, N, s, uu)[-1]
        return 0.5 * np.sum((UN - tgt) ** 2)

    p = orc.Problem(n, a=a, c=0.3, src=src, src_t=src_t)
    J, gu, ga = orc.adjoint(p, T, N, s, u0, tgt)
    assert abs(J - J_of(a, u0)) < 1e-12 * abs(J)
    for d in wl.random_directions(shape_a, 5, 99):
        eps = 1e-5
        fd = (J_of(a + eps * d, u0) - J_of(a - eps * d, u0)) / (2 * eps)
        np.testing.assert_allclose(np.sum(ga * d), fd, rtol=1e-6, atol=1e-10)
    for d in wl.random_directions(n[::-1], 3, 98):
        eps = 1e-2  # J is quadratic in u0: the central difference is exact up to rounding
        fd = (J_of(a, u0 + eps * d) - J_of(a, u0 - eps * d)) / (2 * eps)
        np.testing.assert_allclose(np.sum(gu * d), fd, rtol=1e-7, atol=1e-10)
