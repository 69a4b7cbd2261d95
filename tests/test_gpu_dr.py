"""GPU parity of Parareal/FIE-DR (Sec. 4.2): the fine propagator takes s Douglas-Rachford
steps (eq. DR_method), the coarse one FIE steps.  FP64, with the dimensional splitting and with
the domain-decomposition splitting (Sec. 2.1; Fig. 4 runs FIE-DR with both).

Every call goes through the C ABI.  Results must match the oracle's Parareal/FIE-DR to 1e-12
in relative max-norm with equal iteration counts; the parareal states at n <= k equal the
GPU's own sequential DR solution bitwise (finite termination, Sec. 3).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc

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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def make(ps, n, a=None, c=0.0, src=None, src_t=None, T=1.0, N=4, g=1, s=4, precision="fp64", split="dim",
         boxes=(1, 1), overlap=0.0, coarse=None):
    """coarse = (boxes, overlap) of a separate DD decomposition for G, or None (G uses F's)."""
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=None if a is None else dev(a), c=c, src=None if src is None else dev(src), src_t=src_t)
    sp = ps.Splitting(op, split, boxes, overlap)
    spc = ps.Splitting(op, "dd", coarse[0], coarse[1]) if coarse else None
    prob = ps.Problem(sp, T, N, g, s, coarse=spc, precision=precision, fine_method="dr")
    prob._keep = (grid, op, sp, spc)
    orp = orc.Problem(n, a=a, c=c, src=src, src_t=src_t, split=split, boxes=boxes, overlap=overlap)
    if coarse:
        orp.pG = orc.Problem(n, a=a, c=c, src=src, src_t=src_t, split="dd", boxes=coarse[0], overlap=coarse[1])
    return prob, orp


def inputs(n, N, s, seed):
    rng = np.random.default_rng(seed)
    a = np.exp(0.4 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    src_t = 1.0 + np.sin(np.arange(N * s + 1) * 0.2)
    u0 = rng.standard_normal(n[::-1])
    return a, src, src_t, u0


# (the first three stop before k = N; random data converge slowly under DR, whose factor
# approaches 1 for stiff modes, Theorem 2)
@pytest.mark.parametrize("n,N,s,g,T", [((17, 13), 12, 8, 1, 0.3), ((9, 7, 6), 10, 4, 1, 0.02),
                                       ((40, 3), 10, 6, 2, 0.02), ((1, 5, 2), 3, 3, 1, 0.3)])
def test_parareal_fie_dr_matches_oracle(ps, n, N, s, g, T):
    a, src, src_t, u0 = inputs(n, N, s, 31)
    prob, orp = make(ps, n, a=a, c=0.4, src=src, src_t=src_t, T=T, N=N, g=g, s=s)
    tol = 1e-9
    it = prob.run(dev(u0), tol)
    U_ref, _, it_ref = orc.parareal(orp, T, N, g, s, u0, tol, fine="dr")
    assert it == it_ref
    for j in range(N + 1):
        assert relmax(prob.state(j).cpu().numpy(), U_ref[j]) < RTOL64, j


@pytest.mark.parametrize("n", [(23, 19), (8, 6, 5)])
def test_fine_sequential_dr_matches_oracle(ps, n):
    N, s, T = 4, 5, 0.2
    a, src, src_t, u0 = inputs(n, N, s, 32)
    prob, orp = make(ps, n, a=a, c=0.2, src=src, src_t=src_t, T=T, N=N, s=s)
    got = prob.fine_sequential(dev(u0)).cpu().numpy()
    ref = orc.fine_sequential_dr(orp, T, N, s, u0)
    for j in range(N + 1):
        assert relmax(got[j], ref[j]) < RTOL64, j


def test_constant_coefficient_no_source(ps):
    """a = 1 (no coefficient array), c = 0, no source: the kernels' null-pointer branches."""
    n, N, s, T = (31, 29), 6, 6, 0.5
    rng = np.random.default_rng(33)
    u0 = rng.standard_normal(n[::-1])
    prob, orp = make(ps, n, T=T, N=N, s=s)
    it = prob.run(dev(u0), 1e-10)
    U_ref, _, it_ref = orc.parareal(orp, T, N, 1, s, u0, 1e-10, fine="dr")
    assert it == it_ref
    assert relmax(prob.state(N).cpu().numpy(), U_ref[N]) < RTOL64


def test_finite_termination_bitwise(ps):
    n, N, s = (21, 19), 5, 4
    a, src, src_t, u0 = inputs(n, N, s, 34)
    prob, _ = make(ps, n, a=a, c=0.1, src=src, src_t=src_t, T=0.3, N=N, s=s)
    u0 = dev(u0)
    fine = prob.fine_sequential(u0).cpu().numpy()
    for k in (1, 3, N):
        it = prob.run(u0, 0.0, max_iter=k)
        assert it == k
        for j in range(k + 1):
            assert np.array_equal(prob.state(j).cpu().numpy(), fine[j]), (k, j)


# DD splitting (Sec. 2.1): boxes, overlap in cells, and an optional coarse decomposition
DD_CASES = [((31, 23), (4, 3), 3, None), ((40, 17), (4, 1), 4, ((8, 1), 2)), ((19, 26), (2, 2), 2, None)]


@pytest.mark.parametrize("n,boxes,ovc,coarse", DD_CASES)
def test_parareal_fie_dr_dd_matches_oracle(ps, n, boxes, ovc, coarse):
    N, s, T = 8, 6, 0.25
    a, src, src_t, u0 = inputs(n, N, s, 35)
    h = 1.0 / (max(n) + 1)
    cz = (coarse[0], coarse[1] * h) if coarse else None
    prob, orp = make(ps, n, a=a, c=0.3, src=src, src_t=src_t, T=T, N=N, s=s, split="dd", boxes=boxes,
                     overlap=ovc * h, coarse=cz)
    # thin overlaps contract slowly (Fig. 7): compare the iterate after 3 iterations (every
    # slice past the finite-termination front carries corrections) and the run to k = N
    for max_iter in (3, 0):
        it = prob.run(dev(u0), 1e-9, max_iter)
        U_ref, hist_ref, it_ref = orc.parareal(orp, T, N, 1, s, u0, 1e-9, max_iter=max_iter or None, fine="dr",
                                               pG=getattr(orp, "pG", None))
        assert it == it_ref
        np.testing.assert_allclose(prob.history(), hist_ref, rtol=1e-6)
        for j in range(N + 1):
            assert relmax(prob.state(j).cpu().numpy(), U_ref[j]) < RTOL64, (max_iter, j)


def test_fine_sequential_dr_dd_and_finite_termination(ps):
    n, N, s, T = (29, 21), 5, 4, 0.3
    a, src, src_t, u0 = inputs(n, N, s, 36)
    prob, orp = make(ps, n, a=a, c=0.2, src=src, src_t=src_t, T=T, N=N, s=s, split="dd", boxes=(3, 2),
                     overlap=3.0 / 30)
    u0d = dev(u0)
    fine = prob.fine_sequential(u0d).cpu().numpy()
    ref = orc.fine_sequential_dr(orp, T, N, s, u0)
    for j in range(N + 1):
        assert relmax(fine[j], ref[j]) < RTOL64, j
    for k in (1, 3, N):
        assert prob.run(u0d, 0.0, max_iter=k) == k
        for j in range(k + 1):
            assert np.array_equal(prob.state(j).cpu().numpy(), fine[j]), (k, j)


def test_dr_is_rejected_where_unsupported(ps):
    n = (13, 11)
    with pytest.raises(ps.PsError) as e:
        make(ps, n, precision="mixed")
    assert e.value.code == 6
    prob, _ = make(ps, n, a=np.ones((13, 15)), N=3, s=2)
    u0 = dev(np.ones((11, 13)))
    prob.run(u0, 1e-8)
    with pytest.raises(ps.PsError) as e:
        prob.vjp(prob.state(3), 1e-8)
    assert e.value.code == 6
    with pytest.raises(ps.PsError) as e:
        ps.Batch([prob])
    assert e.value.code == 6
