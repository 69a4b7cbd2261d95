"""The handle calls of the boundary through the C ABI: changing a problem's slice and step
counts (Sec. 3: N, G = g steps, F = s steps per slice), batches built problem by problem with
their states read back through the batch, the adjoint of a target loss, and checkpoint/resume
of a parareal run.

Bars: FP64 states within 1e-12 of the oracle with equal iteration counts; a reconfigured
problem equals a freshly created one bitwise; batched states equal individual runs bitwise;
the target-loss adjoint equals the vector-Jacobian product of U_N - target bitwise and the
oracle's discrete adjoint within 1e-9.
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
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def inputs(n, seed, steps):
    rng = np.random.default_rng(seed)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    src_t = 1.0 + 0.5 * np.sin(0.3 * np.arange(steps + 1))
    u0 = rng.standard_normal(n[::-1])
    return a, src, src_t, u0


@pytest.mark.parametrize("n,split,boxes,ovc", [((33, 27), "dim", (1, 1), 0), ((11, 9, 7), "dim", (1, 1), 0),
                                               ((37, 29), "dd", (3, 3), 3)])
def test_set_slices_matches_oracle_and_fresh_problem(ps, n, split, boxes, ovc):
    T = 0.4
    a, src, src_t, u0 = inputs(n, 51, 8 * 12)
    ov = ovc / (max(n) + 1.0)
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=dev(a), c=0.2, src=dev(src), src_t=src_t)
    sp = ps.Splitting(op, split, boxes, ov)
    prob = ps.Problem(sp, T, 4, 1, 6)
    prob.run(dev(u0), 1e-10)
    # new slice count and step counts, G with two steps per slice
    prob.set_slices(8, 2, 12)
    it = prob.run(dev(u0), 1e-10)
    orp = orc.Problem(n, a=a, c=0.2, src=src, src_t=src_t, split=split, boxes=boxes, overlap=ov)
    U_ref, h_ref, it_ref = orc.parareal(orp, T, 8, 2, 12, u0, 1e-10)
    assert it == it_ref
    np.testing.assert_allclose(prob.history(), h_ref, rtol=1e-6, atol=1e-15)
    for j in range(9):
        assert relmax(prob.state(j).cpu().numpy(), U_ref[j]) < RTOL64, j
    fresh = ps.Problem(sp, T, 8, 2, 12)
    assert fresh.run(dev(u0), 1e-10) == it
    for j in range(9):
        assert torch.equal(fresh.state(j), prob.state(j)), j


def test_set_slices_mixed_forms_and_rejections(ps):
    n, T = (29, 31), 0.5
    a, src, src_t, u0 = inputs(n, 52, 16 * 8)
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=dev(a), src=dev(src), src_t=src_t)
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, T, 4, 1, 4, precision="mixed", coarse_mode="delta32")
    prob.run(dev(u0), 1e-9)
    prob.set_slices(16, 1, 8)
    it = prob.run(dev(u0), 1e-9)
    fresh = ps.Problem(sp, T, 16, 1, 8, precision="mixed", coarse_mode="delta32")
    assert fresh.run(dev(u0), 1e-9) == it
    assert torch.equal(fresh.state(16), prob.state(16))
    # f_steps not a multiple of g_steps, N < 1, a source table too short: refused, nothing changed
    for bad in ((16, 3, 8), (0, 1, 4), (64, 1, 8)):
        with pytest.raises(ps.PsError) as e:
            prob.set_slices(*bad)
        assert e.value.code == 1, bad
    assert prob.run(dev(u0), 1e-9) == it
    assert torch.equal(fresh.state(16), prob.state(16))


def test_batch_add_and_get_state(ps):
    cfgs = wl.batch256(count=5, seed=9, sizes=(17, 31, 47), slices=(4, 8), s_range=(3, 12))

    def make(c):
        grid = ps.Grid(c["n"])
        op = ps.Operator(grid, a=dev(c["a"]))
        sp = ps.Splitting(op)
        p = ps.Problem(sp, c["T"], c["N"], 1, c["s"], precision="mixed")
        p._keep = (grid, op, sp)
        return p

    probs = [make(c) for c in cfgs]
    u0s = [dev(c["u0"]) for c in cfgs]
    ref = []
    for p, u in zip(probs, u0s):
        k = p.run(u, 1e-8)
        ref.append((k, [p.state(n).clone() for n in range(p.N + 1)]))
    batch = ps.Batch([])
    with pytest.raises(ps.PsError) as e:
        batch.run([], 1e-8)
    assert e.value.code == 1
    for p in probs[:2]:
        batch.add(p)
    assert batch.run(u0s[:2], 1e-8) == [r[0] for r in ref[:2]]
    for p in probs[2:]:
        batch.add(p)
    with pytest.raises(ps.PsError) as e:
        batch.add(probs[0])  # already in the batch
    assert e.value.code == 1
    its = batch.run(u0s, 1e-8)
    assert its == [r[0] for r in ref]
    for i, (k, states) in enumerate(ref):
        for n in range(probs[i].N + 1):
            assert torch.equal(batch.state(i, n), states[n]), (i, n)
    with pytest.raises(ps.PsError):
        batch.state(len(probs), 0)
    # a batched problem keeps its slices
    with pytest.raises(ps.PsError) as e:
        probs[0].set_slices(8, 1, 4)
    assert e.value.code == 1


def test_adjoint_of_target_loss(ps):
    n, N, s, T = (19, 15), 4, 6, 0.2
    a, src, src_t, u0 = inputs(n, 53, N * s)
    tgt = np.random.default_rng(54).standard_normal(n[::-1])
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=dev(a), c=0.3, src=dev(src), src_t=src_t)
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, T, N, 1, s, tol_mode=1)
    prob.run(dev(u0), 1e-14)
    J, gu, ga = prob.adjoint(dev(tgt), 1e-14)
    J_ref, gu_ref, ga_ref = orc.adjoint(orc.Problem(n, a=a, c=0.3, src=src, src_t=src_t), T, N, s, u0, tgt)
    assert abs(J - J_ref) <= 1e-10 * J_ref
    assert relmax(gu.cpu().numpy(), gu_ref) < 1e-9
    assert relmax(ga.cpu().numpy(), ga_ref) < 1e-9
    gu2, ga2 = prob.vjp(prob.state(N) - dev(tgt), 1e-14)
    assert torch.equal(gu, gu2) and torch.equal(ga, ga2)
    J2, _, _ = prob.adjoint(dev(tgt), 1e-14)
    assert J2 == J  # fixed summation order


@pytest.mark.parametrize("form", ["fp64", "delta32", "dd"])
def test_checkpoint_resume_is_bitwise_the_uninterrupted_run(ps, form):
    """A run stopped after 3 iterations, saved, loaded into a fresh problem and resumed to the
    tolerance gives the uninterrupted run's iteration count, history and states bitwise; so does
    resuming the stopped problem itself."""
    n, N, s, T = (29, 23), 12, 6, 0.5
    a, src, src_t, u0 = inputs(n, 55, N * s)

    def make():
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), c=0.1, src=dev(src), src_t=src_t)
        sp = ps.Splitting(op, "dd", (3, 2), 3.0 / 30) if form == "dd" else ps.Splitting(op)
        prob = ps.Problem(sp, T, N, 1, s, precision="fp64" if form != "delta32" else "mixed",
                          coarse_mode="delta32" if form == "delta32" else "fp64")
        prob._keep = (grid, op, sp)
        return prob

    tol = 1e-10
    full = make()
    it = full.run(dev(u0), tol)
    assert 3 < it <= N
    ref = ([full.state(j).clone() for j in range(N + 1)], full.history())
    stopped = make()
    assert stopped.run(dev(u0), tol, 3) == 3
    blob = stopped.checkpoint()
    fresh = make()
    fresh.load_checkpoint(blob)
    for prob in (fresh, stopped):
        assert prob.resume(tol) == it
        assert np.array_equal(prob.history(), ref[1])
        for j in range(N + 1):
            assert torch.equal(prob.state(j), ref[0][j]), j
        assert prob.resume(tol) == it  # already converged: no further iteration
    # a checkpoint of another slice count is refused
    other = make()
    other.set_slices(6, 1, 12)
    with pytest.raises(ps.PsError) as e:
        other.load_checkpoint(blob)
    assert e.value.code == 1
    # an edited state is not an iterate to resume
    fresh.set_state(2, fresh.state(2))
    with pytest.raises(ps.PsError):
        fresh.resume(tol)
