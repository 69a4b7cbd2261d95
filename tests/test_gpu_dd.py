"""GPU parity of the domain-decomposition splitting against the FP64 CPU oracle.

The DD substep of colour j solves (I - tau A_j) x = b with A_j built from the
partition of unity rho_j (Sec. 2.1); the GPU factors every box by banded Cholesky
and solves all slices' boxes at once.  FP64 parity bar: 1e-12 relative max-norm,
equal parareal iteration counts.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc
from paper_2502_08370_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
RTOL64 = 1e-12


@pytest.fixture(scope="module")
def ps():
    from paper_2502_08370_gb300 import build
    build.build()
    import paper_2502_08370_gb300 as ps
    return ps


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def relmax(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def make(ps, n, boxes, overlap, a=None, c=0.0, src=None, src_t=None, T=1.0, N=4, g=1, s=4, coarse=None, spb=0):
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=None if a is None else dev(a), c=c, src=None if src is None else dev(src), src_t=src_t)
    sp = ps.Splitting(op, "dd", boxes, overlap)
    spc = ps.Splitting(op, "dd", coarse[0], coarse[1]) if coarse else None
    prob = ps.Problem(sp, T, N, g, s, coarse=spc, dd_slices_per_block=spb)
    prob._keep = (grid, op, sp, spc)
    orp = orc.Problem(n, a=a, c=c, src=src, src_t=src_t, split="dd", boxes=boxes, overlap=overlap)
    orpc = orc.Problem(n, a=a, c=c, src=src, src_t=src_t, split="dd", boxes=coarse[0], overlap=coarse[1]) \
        if coarse else None
    return prob, orp, orpc


CASES = [((31, 23), (4, 3), 3), ((17, 40), (2, 5), 2), ((63, 63), (4, 4), 6), ((30, 9), (5, 1), 2), ((12, 33), (1, 4), 3)]


@pytest.mark.parametrize("n,boxes,ovc", CASES)
def test_dd_substep_matches_oracle(ps, n, boxes, ovc):
    rng = np.random.default_rng(21)
    a = np.exp(0.4 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    ov = ovc / (max(n) + 1.0)
    prob, orp, _ = make(ps, n, boxes, ov, a=a, c=0.7, T=0.6, N=3, s=4)
    b = rng.standard_normal(n[::-1])
    for which, tau in ((0, 0.6 / 3 / 4), (1, 0.6 / 3)):
        for j in range(orp.M):
            x = dev(b)
            prob.substep_solve(which, j, x)
            ref = orc.substep_solve(orp, j, tau, b)
            assert relmax(x.cpu().numpy(), ref) < RTOL64, (which, j)


@pytest.mark.parametrize("spb", [1, 2, 4])
def test_dd_parareal_matches_oracle(ps, spb):
    rng = np.random.default_rng(22)
    n, N, s = (41, 37), 8, 10
    a = np.exp(0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    src = rng.standard_normal(n[::-1])
    src_t = np.cos(0.2 * np.arange(N * s + 1))
    prob, orp, _ = make(ps, n, (4, 4), 4 / 42.0, a=a, c=0.2, src=src, src_t=src_t, T=0.5, N=N, g=1, s=s, spb=spb)
    u0 = rng.standard_normal(n[::-1])
    it = prob.run(dev(u0), 1e-10)
    U_ref, h_ref, it_ref = orc.parareal(orp, 0.5, N, 1, s, u0, 1e-10)
    assert it == it_ref
    np.testing.assert_allclose(prob.history(), h_ref, rtol=1e-6, atol=1e-15)
    for j in range(N + 1):
        assert relmax(prob.state(j).cpu().numpy(), U_ref[j]) < RTOL64, j


def test_dd_different_coarse_and_fine_decompositions(ps):
    """Sec. 5.1's setting: strips, G with q = 4 / beta = 1/32, F with q = 2 / beta = 1/16."""
    n, T, N, s = (49, 49), 1.0, 8, 10
    S, st, _ = wl.manufactured(n, T, N, s)
    prob, orp, orpc = make(ps, n, (4, 1), 1 / 16, src=S, src_t=st, T=T, N=N, g=1, s=s, coarse=((8, 1), 1 / 32))
    u0 = np.zeros(n[::-1])
    it = prob.run(dev(u0), 0.0, max_iter=4)
    U_ref, _, it_ref = orc.parareal(orp, T, N, 1, s, u0, 0.0, max_iter=4, pG=orpc)
    assert it == it_ref == 4
    for j in range(N + 1):
        assert relmax(prob.state(j).cpu().numpy(), U_ref[j]) < RTOL64, j


def test_dd_finite_termination_bitwise(ps):
    rng = np.random.default_rng(23)
    n, N, s = (33, 29), 5, 4
    prob, _, _ = make(ps, n, (3, 3), 3 / 34.0, T=0.3, N=N, s=s)
    u0 = dev(rng.standard_normal(n[::-1]))
    fine = prob.fine_sequential(u0).cpu().numpy()
    for k in (1, 3, N):
        prob.run(u0, 0.0, max_iter=k)
        for j in range(k + 1):
            assert np.array_equal(prob.state(j).cpu().numpy(), fine[j]), (k, j)


def test_dd2d_1023_full_size_substeps_and_run(ps):
    """1023^2, 8x8 boxes, overlap 8 cells: every colour's substep equals the oracle's on the
    full grid; a fixed number of parareal iterations (the paper's DD scalability runs use 5;
    with this thin overlap the increments do not contract monotonically, in the oracle too)
    keeps the finite-termination property: U_1 = F(u0) bitwise."""
    cfg = wl.dd2d_1023()
    n = cfg["n"]
    prob, orp, _ = make(ps, n, cfg["boxes"], cfg["overlap"], T=cfg["T"], N=cfg["N"], g=1, s=cfg["s"])
    u0 = cfg["u0"]
    tau_f = cfg["T"] / cfg["N"] / cfg["s"]
    for j in range(4):
        x = dev(u0)
        prob.substep_solve(0, j, x)
        ref = orc.substep_solve(orp, j, tau_f, u0)
        assert relmax(x.cpu().numpy(), ref) < RTOL64, j
    u0d = dev(u0)
    it = prob.run(u0d, 0.0, max_iter=2)
    hist = prob.history()
    assert it == 2 and all(np.isfinite(hist))
    # U_1 of the final iterate is exactly F(u0): compare with a GPU fine propagation of u0
    x = dev(u0)
    prob.propagate(0, cfg["s"], x, t0=0, tstride=1)
    assert np.array_equal(prob.state(1).cpu().numpy(), x.cpu().numpy())


def test_dd_autotune_slices_per_cta_changes_no_result(ps):
    """The autotuner picks the time slices per CTA of the colour solves; every slice's arithmetic
    is the same for any count, so the states stay bitwise equal."""
    rng = np.random.default_rng(24)
    n, N, s = (41, 37), 10, 6
    a = np.exp(0.3 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    prob, _, _ = make(ps, n, (4, 4), 4 / 42.0, a=a, T=0.5, N=N, s=s, spb=1)
    u0 = dev(rng.standard_normal(n[::-1]))
    it = prob.run(u0, 1e-10)
    before = [prob.state(j).cpu().numpy() for j in range(N + 1)]
    choice = prob.autotune(budget_ms=20)
    assert choice in (1, 2, 4)
    rec = prob.autotune_record()
    assert sorted(r[0] for r in rec) == ["dd:1-slices-per-cta", "dd:2-slices-per-cta", "dd:4-slices-per-cta"]
    assert sum(r[2] for r in rec) == 1
    assert prob.run(u0, 1e-10) == it
    for j in range(N + 1):
        assert np.array_equal(prob.state(j).cpu().numpy(), before[j]), j
