"""GPU adjoint (vector-Jacobian product) against the oracle's discrete adjoint and against
central finite differences of the GPU forward solve.

J = 1/2 ||U_N - target||^2 with U_N the sequential fine solution (the parareal run is
taken to a tight per-slice relative tolerance so that its U_N equals the fine solution to
~1e-13).  Bars: oracle adjoint 1e-9 relative max-norm (parareal, not sequential, on the
GPU side); finite differences 1e-6 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2502_08370_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    from paper_2502_08370_gb300 import build
    build.build()
    import paper_2502_08370_gb300 as ps
    return ps


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def relmax(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def build(ps, n, a, c=0.0, src=None, src_t=None, T=0.2, N=4, s=6, g=1):
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=dev(a), c=c, src=None if src is None else dev(src), src_t=src_t)
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, T, N, g, s, tol_mode=1)
    prob._keep = (grid, op, sp)
    return prob


@pytest.mark.parametrize("n,N,s,g", [((13, 11), 4, 6, 1), ((9, 7, 6), 3, 4, 2), ((40, 33), 6, 8, 1)])
def test_adjoint_matches_oracle(ps, n, N, s, g):
    rng = np.random.default_rng(41)
    shape_a = tuple(v + 2 for v in reversed(n))
    a = np.exp(0.3 * rng.standard_normal(shape_a))
    src = rng.standard_normal(n[::-1])
    T = 0.2
    src_t = 1.0 + 0.5 * np.sin(np.arange(N * s + 1) * 0.7)
    u0 = rng.standard_normal(n[::-1])
    tgt = rng.standard_normal(n[::-1])
    prob = build(ps, n, a, c=0.3, src=src, src_t=src_t, T=T, N=N, s=s, g=g)
    prob.run(dev(u0), 1e-14)
    UN = prob.state(N)
    gN = UN - dev(tgt)
    gu, ga = prob.vjp(gN, 1e-14)
    orp = orc.Problem(n, a=a, c=0.3, src=src, src_t=src_t)
    J, gu_ref, ga_ref = orc.adjoint(orp, T, N, s, u0, tgt)
    assert abs(0.5 * float((gN ** 2).sum()) - J) <= 1e-10 * abs(J)
    assert relmax(gu.cpu().numpy(), gu_ref) < 1e-9
    assert relmax(ga.cpu().numpy(), ga_ref) < 1e-9
    # the problem's states are the forward states again
    assert torch.equal(prob.state(N), UN)


def test_adjoint_finite_differences_adjoint2d(ps):
    """The adjoint workload's recipe at reduced size: 20 seeded unit directions for a,
    5 for u0; central differences of J from the GPU forward solve."""
    cfg = wl.adjoint2d_511(n=63, N=8, s=16)
    n = cfg["n"]
    prob = build(ps, n, cfg["a"], T=cfg["T"], N=cfg["N"], s=cfg["s"])
    u0 = dev(cfg["u0"])
    # target: the fine solution of the perturbed coefficient
    prob.update_coefficients(dev(cfg["a_target"]))
    prob.run(u0, 1e-14)
    tgt = prob.state(cfg["N"]).clone()
    a = dev(cfg["a"])

    def J_of(aa, uu):
        prob.update_coefficients(aa)
        prob.run(uu, 1e-14)
        d = prob.state(cfg["N"]) - tgt
        return 0.5 * float((d * d).sum())

    J0 = J_of(a, u0)
    gN = prob.state(cfg["N"]) - tgt
    gu, ga = prob.vjp(gN, 1e-14)
    assert J0 > 0
    for d in wl.random_directions(tuple(a.shape), 20, cfg["dirs_seed"]):
        dd = dev(d)
        eps = 1e-4
        fd = (J_of(a + eps * dd, u0) - J_of(a - eps * dd, u0)) / (2 * eps)
        an = float((ga * dd).sum())
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-30, (an, fd)
    for d in wl.random_directions(tuple(u0.shape), 5, cfg["dirs_seed"] + 1):
        dd = dev(d)
        eps = 1e-3
        fd = (J_of(a, u0 + eps * dd) - J_of(a, u0 - eps * dd)) / (2 * eps)
        an = float((gu * dd).sum())
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-30, (an, fd)


def test_adjoint_full_size_directional_derivatives(ps):
    """511^2, N = 32, s = 64: <grad, d> against fourth-order central differences of J on all
    20 seeded unit directions of a and 5 of u0, J evaluated on the discrete forward map the
    adjoint differentiates (N*s fine steps from u0).  The gradient compared is the exact one of
    that map: forward and adjoint parareal run to k = N (finite termination, Sec. 3), so the
    only differences left are the finite differences' own.  U_N's ~1e-15 relative rounding,
    divided by e, limits small steps; on a direction whose derivative is far below the median,
    the fourth-order stencil at e = 0.1 missed by 1.35e-6 and its value at e = 0.05 by twice as
    much (noise, not truncation).  The stencils at e = 0.4 and 0.2 are combined to sixth order
    (each node then moves by ~8e-4).  The gradient at the workload's
    tolerance 1e-10 is compared with the exact one as well."""
    cfg = wl.adjoint2d_511()
    n, N = cfg["n"], cfg["N"]
    prob = build(ps, n, cfg["a"], T=cfg["T"], N=N, s=cfg["s"])
    u0 = dev(cfg["u0"])
    prob.update_coefficients(dev(cfg["a_target"]))
    tgt = prob.fine_sequential(u0)[N].clone()
    a = dev(cfg["a"])
    prob.update_coefficients(a)
    prob.run(u0, cfg["tol"])
    gu_tol, ga_tol = prob.vjp(prob.state(N) - tgt, cfg["tol"])
    prob.run(u0, 0.0)  # k = N: U_N is the sequential fine solution
    gN = prob.state(N) - tgt
    gu, ga = prob.vjp(gN, 0.0)
    # the workload's tolerance moves the gradient by little more than the tolerance itself
    assert relmax(ga_tol.cpu().numpy(), ga.cpu().numpy()) < 1e-7
    assert relmax(gu_tol.cpu().numpy(), gu.cpu().numpy()) < 1e-7

    def J_of(aa, uu):
        prob.update_coefficients(aa)
        x = uu.clone()
        prob.propagate(0, N * cfg["s"], x)
        r = x - tgt
        return 0.5 * float((r * r).sum())

    def fd6(f, eps):
        # fourth-order central differences at eps and eps/2, Richardson-extrapolated to sixth
        # order (their eps^4 truncation terms cancel); J at +-eps is shared by both
        memo = {}

        def F(e):
            if e not in memo:
                memo[e] = f(e)
            return memo[e]

        def fd4(h):
            return (8.0 * (F(h) - F(-h)) - (F(2 * h) - F(-2 * h))) / (12.0 * h)

        return (16.0 * fd4(eps / 2) - fd4(eps)) / 15.0

    # e = 0.4: the rounding noise of the J differences falls as 1/e, and the sixth-order
    # combination keeps the truncation small there (J is smooth in the direction's amplitude)
    eps = 0.4
    rows = []
    for d in wl.random_directions(tuple(a.shape), 20, cfg["dirs_seed"]):
        dd = dev(d)
        fd = fd6(lambda e: J_of(a + e * dd, u0), eps)
        an = float((ga * dd).sum())
        rows.append((an, fd))
    import json
    import os
    rec = os.environ.get("PS_TEST_RECORD")
    if rec:
        with open(rec, "a") as f:
            f.write(json.dumps({"test": "adjoint511_fd_a", "eps": eps, "adjoint_vs_fd6": rows}) + "\n")
    for an, fd in rows:
        assert abs(an - fd) <= 1e-6 * abs(fd), (an, fd)
    for d in wl.random_directions(tuple(u0.shape), 5, cfg["dirs_seed"] + 1):
        dd = dev(d)
        fd = fd6(lambda e: J_of(a, u0 + e * dd), eps)
        an = float((gu * dd).sum())
        assert abs(an - fd) <= 1e-6 * abs(fd), (an, fd)


def test_adjoint_full_size_matches_oracle(ps):
    """511^2, N = 32, s = 64: the GPU gradient (parareal forward and adjoint to 1e-10 per-slice
    relative) against the oracle's sequential discrete adjoint, for J = 1/2 ||U_N||^2."""
    cfg = wl.adjoint2d_511()
    n, N = cfg["n"], cfg["N"]
    prob = build(ps, n, cfg["a"], T=cfg["T"], N=N, s=cfg["s"])
    prob.run(dev(cfg["u0"]), cfg["tol"])
    UN = prob.state(N)
    gu, ga = prob.vjp(UN, cfg["tol"])
    J, gu_ref, ga_ref = orc.adjoint(orc.Problem(n, a=cfg["a"]), cfg["T"], N, cfg["s"], cfg["u0"],
                                    np.zeros(n[::-1]))
    assert abs(0.5 * float((UN * UN).sum()) - J) <= 1e-10 * J
    assert relmax(gu.cpu().numpy(), gu_ref) < 1e-9
    assert relmax(ga.cpu().numpy(), ga_ref) < 1e-9


def test_autograd_function(ps):
    rng = np.random.default_rng(43)
    n, N, s = (21, 17), 4, 8
    shape_a = tuple(v + 2 for v in reversed(n))
    a0 = np.exp(0.2 * rng.standard_normal(shape_a))
    prob = build(ps, n, a0, T=0.1, N=N, s=s)
    u0 = dev(rng.standard_normal(n[::-1])).requires_grad_(True)
    a = dev(a0).requires_grad_(True)
    tgt = dev(rng.standard_normal(n[::-1]))
    UN = ps.parareal_solve(prob, u0, a, 1e-14)
    loss = 0.5 * ((UN - tgt) ** 2).sum()
    loss.backward()
    orp = orc.Problem(n, a=a0)
    J, gu_ref, ga_ref = orc.adjoint(orp, 0.1, N, s, u0.detach().cpu().numpy(), tgt.cpu().numpy())
    assert abs(float(loss.detach()) - J) <= 1e-10 * J
    assert relmax(u0.grad.cpu().numpy(), gu_ref) < 1e-9
    assert relmax(a.grad.cpu().numpy(), ga_ref) < 1e-9


@pytest.mark.parametrize("n", [(300, 11), (9, 280)])
def test_adjoint_long_lines_matches_oracle(ps, n):
    rng = np.random.default_rng(44)
    shape_a = tuple(v + 2 for v in reversed(n))
    a = np.exp(0.3 * rng.standard_normal(shape_a))
    N, s, T = 2, 3, 0.01
    u0 = rng.standard_normal(n[::-1])
    tgt = rng.standard_normal(n[::-1])
    prob = build(ps, n, a, T=T, N=N, s=s)
    prob.run(dev(u0), 1e-14)
    gN = prob.state(N) - dev(tgt)
    gu, ga = prob.vjp(gN, 1e-14)
    J, gu_ref, ga_ref = orc.adjoint(orc.Problem(n, a=a), T, N, s, u0, tgt)
    assert relmax(gu.cpu().numpy(), gu_ref) < 1e-9
    assert relmax(ga.cpu().numpy(), ga_ref) < 1e-9


def oracle_u0_gradient(orp, orp_nosrc, T, N, s, u0, tgt):
    """dJ/du0 for J = 1/2 ||U_N - target||^2 with U_N the sequential fine solution: every FIE
    substep solve is symmetric, so the transposed fine step is the step's substeps in reverse
    order without the source, applied to U_N - target from the last step to the first."""
    U = orc.fine_sequential(orp, T, N, s, u0)
    lam = U[N] - tgt
    tau = T / N / s
    for _ in range(N * s):
        lam = orc.fie_step(orp_nosrc, tau, lam, reversed_order=True)
    return 0.5 * float(np.sum((U[N] - tgt) ** 2)), lam


@pytest.mark.parametrize("form", ["mixed", "dd"])
def test_u0_gradient_fp32_form_and_dd_splitting(ps, form):
    """dJ/du0 through the adjoint parareal in the FP32 form (FP32 fine line solves) and with the
    DD splitting (FP64): against the transposed oracle fine propagator, itself pinned here by a
    central difference of the quadratic J (exact up to rounding).  Bars: the FP32 bound of the
    forward solve (4 s N M 2^-24, relative to max |dJ/du0|); 1e-9 in FP64.  The coefficient
    gradient of these forms is refused (PS_ERR_UNSUPPORTED)."""
    n, N, s, T = (23, 19), 4, 5, 0.3
    rng = np.random.default_rng(81)
    a = np.exp(0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    src = rng.standard_normal(n[::-1])
    src_t = 1.0 + 0.2 * np.sin(np.arange(N * s + 1))
    u0 = rng.standard_normal(n[::-1])
    tgt = rng.standard_normal(n[::-1])
    split, boxes, ov = ("dd", (3, 2), 3.0 / 24) if form == "dd" else ("dim", (1, 1), 0.0)
    orp = orc.Problem(n, a=a, src=src, src_t=src_t, split=split, boxes=boxes, overlap=ov)
    orp0 = orc.Problem(n, a=a, split=split, boxes=boxes, overlap=ov)
    J_ref, g_ref = oracle_u0_gradient(orp, orp0, T, N, s, u0, tgt)
    # pin: J is quadratic in u0, so the central difference is exact up to rounding
    d = rng.standard_normal(n[::-1])
    eps = 1e-3
    Jp = 0.5 * np.sum((orc.fine_sequential(orp, T, N, s, u0 + eps * d)[N] - tgt) ** 2)
    Jm = 0.5 * np.sum((orc.fine_sequential(orp, T, N, s, u0 - eps * d)[N] - tgt) ** 2)
    assert abs((Jp - Jm) / (2 * eps) - np.sum(g_ref * d)) <= 1e-8 * abs(np.sum(g_ref * d))
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=dev(a), src=dev(src), src_t=src_t)
    sp = ps.Splitting(op, split, boxes, ov)
    prob = ps.Problem(sp, T, N, 1, s, tol_mode=1, precision="mixed" if form == "mixed" else "fp64")
    prob.run(dev(u0), 1e-13)
    J, gu, _ = prob.adjoint(dev(tgt), 1e-13, want_a=False)
    bar = 4.0 * s * N * 2 * 2.0 ** -24 if form == "mixed" else 1e-9
    assert abs(J - J_ref) <= bar * J_ref * 10
    assert relmax(gu.cpu().numpy(), g_ref) < bar
    with pytest.raises(ps.PsError) as e:
        prob.adjoint(dev(tgt), 1e-13, want_a=True)
    assert e.value.code == 6
