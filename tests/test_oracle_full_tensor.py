"""Pins of the oracle's full-diffusion-tensor operator (Sec. 5.2), CPU only.

D = [[d11, d12], [d12, d22]] with d11 = d22 = 1/(2 + cos(3 pi x) cos(2 pi y)), d12 = 1/4 (the
paper's tensor).  The mixed derivatives rule out dimensional splitting (Sec. 2.1), so only
the DD splitting takes it; the discrete operator has a 9-point stencil.

- The closed form of div(D grad S) used as the analytic reference is checked symbolically.
- Consistency: the unsplit discrete operator applied to S = sin(2 pi x) sin(2 pi y) approaches
  div(D grad S) at second order in h.  A wrong sign, factor or index of the mixed term leaves
  an O(1) error.
- Every A_j is symmetric with a 9-point stencil, -A_j is positive semidefinite, and the A_j sum
  to the unsplit operator.
- Each DD substep equals (I - tau A_j)^{-1} b evaluated densely.  This covers the box
  assembly, the band widened for the corner couplings, and the box ranges.  At large tau
  the box Cholesky still succeeds.  A mixed term discretised at the nodes next to edge-based
  diagonal fluxes fails there: its A_j are indefinite inside the overlaps.
- The fine solution of the manufactured problem converges to the exact solution: first order
  in time for FIE.
- Parareal/FIE-FIE and FIE-DR terminate bitwise at k = N.  Sec. 5.2 (Fig. 10): FIE-FIE
  converges faster for smaller s; FIE-DR deteriorates at s = 2 and behaves alike for s >= 4.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2502_08370_gb300 import workloads as wl


def axis(n):
    return np.arange(1, n + 1) / (n + 1.0)


def tensor_problem(n, boxes=(1, 1), overlap=0.0, d12=None, T=1.0, N=4, s=4, with_source=False):
    m = wl.manufactured_full_tensor(n, T, N, s)
    kw = dict(src=m["src"], src_t=m["src_t"], src2=m["src2"], src2_t=m["src2_t"]) if with_source else {}
    return orc.Problem(n, a=m["a"], d12=m["d12"] if d12 is None else d12, split="dd", boxes=boxes,
                       overlap=overlap, **kw), m


def dense_ops(p, n):
    size = n[0] * n[1]
    out = []
    e = np.zeros(size)
    for j in range(p.M):
        A = np.zeros((size, size))
        for c in range(size):
            e[:] = 0.0
            e[c] = 1.0
            A[:, c] = orc.apply_A(p, j, e.reshape(n[::-1])).reshape(-1)
        out.append(A)
    return out


def test_closed_form_of_the_analytic_operator():
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    d = 1 / (2 + sp.cos(3 * sp.pi * x) * sp.cos(2 * sp.pi * y))
    S = sp.sin(2 * sp.pi * x) * sp.sin(2 * sp.pi * y)
    b = sp.Rational(1, 4)
    L = sp.diff(d * sp.diff(S, x) + b * sp.diff(S, y), x) + sp.diff(b * sp.diff(S, x) + d * sp.diff(S, y), y)
    f = sp.lambdify((x, y), L, "numpy")
    xs, ys = np.array([0.13, 0.5, 0.77, 0.91]), np.array([0.21, 0.38, 0.64])
    got = wl.full_tensor_div_grad_S(xs, ys)
    ref = f(*np.meshgrid(xs, ys))
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_mixed_term_second_order_consistent():
    errs = []
    for n in (63, 127, 255):
        p, _ = tensor_problem((n, n))
        x = axis(n)
        S = np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x))
        got = orc.apply_A(p, 0, S)
        ref = wl.full_tensor_div_grad_S(x, x)
        errs.append(np.abs(got - ref).max() / np.abs(ref).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 < r < 2.1 for r in rates), (errs, rates)
    # without the mixed term the same operator misses div(D grad S) by O(1)
    p0, _ = tensor_problem((31, 31), d12=0.0)
    x = axis(31)
    S = np.outer(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x))
    ref = wl.full_tensor_div_grad_S(x, x)
    assert np.abs(orc.apply_A(p0, 0, S) - ref).max() > 0.05 * np.abs(ref).max()


@pytest.mark.parametrize("n,boxes,overlap", [((9, 8), (2, 2), 2.0 / 10), ((15, 7), (4, 1), 1.0 / 16),
                                             ((12, 11), (3, 3), 1.0 / 13)])
def test_split_operators_symmetric_nine_point_and_summing_to_a(n, boxes, overlap):
    rng = np.random.default_rng(40)
    d12 = 0.25 * (1.0 + 0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    p, _ = tensor_problem(n, boxes, overlap, d12=d12)
    p1, _ = tensor_problem(n, d12=d12)
    mats = dense_ops(p, n)
    (A,) = dense_ops(p1, n)
    scale = np.abs(A).max()
    assert np.abs(sum(mats) - A).max() <= 1e-13 * scale
    ii, jj = np.meshgrid(np.arange(n[0]), np.arange(n[1]))
    ii, jj = ii.ravel(), jj.ravel()
    far = (np.abs(ii[:, None] - ii[None, :]) > 1) | (np.abs(jj[:, None] - jj[None, :]) > 1)
    corner = (np.abs(ii[:, None] - ii[None, :]) == 1) & (np.abs(jj[:, None] - jj[None, :]) == 1)
    for Aj in mats + [A]:
        assert np.abs(Aj - Aj.T).max() <= 1e-13 * scale
        assert not np.any(Aj[far])
        assert np.linalg.eigvalsh(-Aj).min() >= -1e-10 * scale
    assert np.any(A[corner])  # the mixed derivatives are there
    assert np.linalg.eigvalsh(-A).min() > 0


@pytest.mark.parametrize("n,boxes,overlap", [((9, 8), (2, 2), 2.0 / 10), ((15, 7), (4, 1), 1.0 / 16),
                                             ((12, 11), (3, 3), 1.0 / 13), ((31, 9), (8, 1), 1.0 / 32)])
def test_dd_substep_matches_dense_solve(n, boxes, overlap):
    rng = np.random.default_rng(41)
    p, _ = tensor_problem(n, boxes, overlap)
    mats = dense_ops(p, n)
    I = np.eye(n[0] * n[1])
    for tau in (0.003, 0.2):
        for j, Aj in enumerate(mats):
            b = rng.standard_normal(n[::-1])
            got = orc.substep_solve(p, j, tau, b)
            ref = np.linalg.solve(I - tau * Aj, b.reshape(-1)).reshape(n[::-1])
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (j, tau)
    # large steps: I - tau A_j stays SPD (A_j is semidefinite), so the box Cholesky succeeds;
    # checked by the residual, the solution itself being ill-conditioned there
    for j, Aj in enumerate(mats):
        b = rng.standard_normal(n[::-1]).reshape(-1)
        got = orc.substep_solve(p, j, 50.0, b.reshape(n[::-1])).reshape(-1)
        res = (I - 50.0 * Aj) @ got - b
        assert np.abs(res).max() <= 1e-9 * (1 + 50.0 * np.abs(Aj).sum(1).max()) * np.abs(b).max(), j


def test_d12_needs_the_dd_splitting():
    with pytest.raises(ValueError):
        orc.Problem((5, 5), d12=0.25)
    with pytest.raises(ValueError):
        orc.Problem((4, 4, 4), d12=0.25, split="dd", boxes=(2, 2))


def fine_error(p, m, n, T, N, s, fine="fie"):
    h = 1.0 / (n + 1)
    u0 = np.zeros((n, n))
    U = orc.fine_sequential_dr(p, T, N, s, u0) if fine == "dr" else orc.fine_sequential(p, T, N, s, u0)
    return max(np.sqrt(h * h * np.sum((U[j] - m["exact"](j * T / N)) ** 2)) for j in range(1, N + 1))


@pytest.mark.slow
def test_manufactured_fine_solution_first_order_in_time():
    n, T, N = 63, 1.0, 20
    errs = []
    for s in (5, 10, 20):
        p, m = tensor_problem((n, n), (4, 1), 1.0 / 16, T=T, N=N, s=s, with_source=True)
        errs.append(fine_error(p, m, n, T, N, s))
    r = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(1.6 < v < 2.2 for v in r), (errs, r)


@pytest.mark.parametrize("fine", ["fie", "dr"])
def test_parareal_full_tensor_finite_termination_bitwise(fine):
    n, T, N, s = (13, 11), 0.5, 4, 3
    rng = np.random.default_rng(42)
    p, _ = tensor_problem(n, (4, 1), 1.0 / 12, T=T, N=N, s=s, with_source=True)
    u0 = rng.standard_normal(n[::-1])
    F = orc.fine_sequential_dr(p, T, N, s, u0) if fine == "dr" else orc.fine_sequential(p, T, N, s, u0)
    U, _, it = orc.parareal(p, T, N, 1, s, u0, 0.0, max_iter=N, fine=fine)
    assert it == N
    for j in range(N + 1):
        assert np.array_equal(U[j], F[j]), j


@pytest.mark.slow
def test_fig10_dependence_on_s():
    """Errors against the fine solution after k iterations, manufactured problem, h = 1/32,
    Delta T = 0.05, two subdomains of one strip each with beta = 1/16."""
    n, T, N = 31, 1.0, 20
    h = 1.0 / (n + 1)

    def err(fine, s, k):
        p, _ = tensor_problem((n, n), (2, 1), 1.0 / 16, T=T, N=N, s=s, with_source=True)
        u0 = np.zeros((n, n))
        F = orc.fine_sequential_dr(p, T, N, s, u0) if fine == "dr" else orc.fine_sequential(p, T, N, s, u0)
        U, _, _ = orc.parareal(p, T, N, 1, s, u0, 0.0, max_iter=k, fine=fine)
        return max(np.sqrt(h * h * np.sum((U[j] - F[j]) ** 2)) for j in range(1, N + 1))

    fie = [err("fie", s, 4) for s in (2, 4, 10)]
    assert fie[0] < fie[1] < fie[2], fie
    dr = {s: (err("dr", s, 5), err("dr", s, 6)) for s in (2, 4, 10)}
    assert dr[2][1] / dr[2][0] > 0.6  # s = 2: no exponential decay
    assert all(dr[s][1] / dr[s][0] < 0.45 for s in (4, 10)), dr
    assert dr[4][1] / dr[10][1] < 10 and dr[10][1] / dr[4][1] < 10, dr


def test_fie_step_with_two_source_terms_matches_dense_definition():
    """eq. FIE_method with f = src src_t + src2 src2_t: V_0 = U + tau f(t_end), then the colour
    solves in order, evaluated with dense matrices."""
    n = (11, 9)
    rng = np.random.default_rng(43)
    src2, src2_t = rng.standard_normal(n[::-1]), np.cos(np.arange(12) * 0.4)
    m = wl.manufactured_full_tensor(n, 1.0, 3, 3)
    p = orc.Problem(n, a=m["a"], d12=m["d12"], c=0.3, src=m["src"], src_t=m["src_t"], src2=src2, src2_t=src2_t,
                    split="dd", boxes=(2, 2), overlap=2.0 / 12)
    mats = dense_ops(p, n)
    I = np.eye(n[0] * n[1])
    u = rng.standard_normal(n[::-1])
    tau, t_end = 0.07, 5
    v = (u + tau * m["src"] * m["src_t"][t_end] + tau * src2 * src2_t[t_end]).reshape(-1)
    for Aj in mats:
        v = np.linalg.solve(I - tau * Aj, v)
    got = orc.fie_step(p, tau, u, t_end=t_end).reshape(-1)
    assert np.abs(got - v).max() <= 1e-12 * np.abs(v).max()
