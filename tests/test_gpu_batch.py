"""Batched problems (grouped launches, CUDA graph per iteration) and the schedule autotuner.

A batch must reproduce each problem's own ps_run_parareal bitwise (same arithmetic per
line, only the launch grouping differs); the autotuner changes the tile schedule and
therefore must not change any result either.  One problem of the small batch is also
checked against the FP64 oracle within the FP32 line-solve bound.
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


def make(ps, cfg):
    grid = ps.Grid(cfg["n"])
    op = ps.Operator(grid, a=None if cfg["a"] is None else dev(cfg["a"]))
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, cfg["T"], cfg["N"], 1, cfg["s"], precision="mixed")
    prob._keep = (grid, op, sp)
    return prob


def small_batch(count=7, seed=5):
    return wl.batch256(count=count, seed=seed, sizes=(17, 31, 47, 64), slices=(4, 8, 16), s_range=(3, 20))


def snapshot(prob):
    return [prob.state(n).cpu().numpy() for n in range(prob.N + 1)]


def test_small_batch_equals_individual_runs_bitwise(ps):
    cfgs = small_batch()
    probs = [make(ps, c) for c in cfgs]
    u0s = [dev(c["u0"]) for c in cfgs]
    ref_it, ref_states, ref_hist = [], [], []
    for p, u in zip(probs, u0s):
        ref_it.append(p.run(u, 1e-8))
        ref_states.append(snapshot(p))
        ref_hist.append(p.history())
    batch = ps.Batch(probs)
    its = batch.run(u0s, 1e-8)
    assert its == ref_it
    for p, st, h in zip(probs, ref_states, ref_hist):
        got = snapshot(p)
        for n in range(p.N + 1):
            assert np.array_equal(got[n], st[n]), n
        assert np.array_equal(p.history(), h)
    # a second run of the same batch (graphs re-used) gives the same again
    its2 = batch.run(u0s, 1e-8)
    assert its2 == ref_it
    assert np.array_equal(snapshot(probs[0])[-1], ref_states[0][-1])
    # one problem against the FP64 oracle, within the FP32 line-solve bound
    c = cfgs[0]
    U_ref, _, _ = orc.parareal(orc.Problem(c["n"], a=c["a"]), c["T"], c["N"], 1, c["s"], c["u0"], 1e-8)
    err = np.abs(ref_states[0][-1] - U_ref[-1]).max() / np.abs(U_ref[-1]).max()
    assert err < 4.0 * c["s"] * c["N"] * 2 * 2.0 ** -24


def test_autotune_changes_no_result(ps):
    """In a batch (FP64 coarse propagator) the autotuner only weighs schedules with the same
    arithmetic per line: the tile shapes, staged or streamed coarse sweeps, Thomas for the coarse
    x-sweep.  The problem's results stay bitwise the same."""
    c = wl.batch256(count=1, seed=11, sizes=(127,), slices=(32,), s_range=(16, 16))[0]
    p = make(ps, c)
    u0 = dev(c["u0"])
    p.run(u0, 1e-8)
    before = snapshot(p)
    batch = ps.Batch([p])
    choice = p.autotune(budget_ms=50)
    assert choice > 0
    assert all(not r[0].startswith("coarse-x64:") or r[0].endswith("thomas") for r in p.autotune_record())
    p.run(u0, 1e-8)
    after = snapshot(p)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    del batch


def test_autotune_outside_a_batch_may_change_roundings_only(ps):
    """Alone, the FP64 coarse x-sweep may take the hybrid schedule: the coarse values change at
    FP64 rounding, the converged states stay within the tolerance of the same fixed point."""
    c = wl.batch256(count=1, seed=12, sizes=(255,), slices=(16,), s_range=(16, 16))[0]
    p = make(ps, c)
    u0 = dev(c["u0"])
    it = p.run(u0, 1e-10)
    before = snapshot(p)
    p.autotune(budget_ms=50)
    names = [r[0] for r in p.autotune_record()]
    assert {"coarse-x64:thomas", "coarse-x64:hybrid", "coarse-corr:fused", "coarse-corr:split"} <= set(names)
    assert p.run(u0, 1e-10) == it
    after = snapshot(p)
    for a, b in zip(before, after):
        assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()


def test_batch256_sampled_against_individual_runs(ps):
    """The full heterogeneous batch (256 problems, grids up to 511^2, N up to 64, s up to 128):
    eight sampled problems re-run alone must match their batched results bitwise, and on each of
    them a sampled slice of the converged batched iterate satisfies U_{j+1} ~ F(U_j) against the
    oracle's FP64 fine steps, within the FP32 bound of one slice (4 s M 2^-24) plus twice the
    problem's last increment (F and G are max-norm contractions); U_1 = F(u0) within the FP32
    bound (finite termination)."""
    cfgs = wl.batch256()
    probs = [make(ps, c) for c in cfgs]
    u0s = [dev(c["u0"]) for c in cfgs]
    batch = ps.Batch(probs)
    its = batch.run(u0s, 1e-8)
    assert all(1 <= k <= c["N"] for k, c in zip(its, cfgs))
    rng = np.random.default_rng(0)
    sample = [int(i) for i in rng.choice(len(cfgs), 8, replace=False)]
    batched = {i: (its[i], [batch.state(i, j).cpu().numpy() for j in range(cfgs[i]["N"] + 1)],
                   probs[i].history()) for i in sample}
    for i in sample:
        c = cfgs[i]
        k, U, hist = batched[i]
        bound = 4.0 * c["s"] * 2 * 2.0 ** -24
        orp = orc.Problem(c["n"], a=c["a"])
        tau = c["T"] / c["N"] / c["s"]
        u1 = orc.propagate(orp, tau, c["s"], c["u0"], t0=0, tstride=1)
        assert np.abs(U[1] - u1).max() <= bound * np.abs(u1).max(), i
        j = int(rng.integers(k, c["N"])) if k < c["N"] else c["N"] - 1
        ref = orc.propagate(orp, tau, c["s"], U[j], t0=j * c["s"], tstride=1)
        assert np.abs(U[j + 1] - ref).max() <= bound * np.abs(ref).max() + 2 * hist[-1], (i, j)
    for i in sample:
        k = probs[i].run(u0s[i], 1e-8)
        assert k == batched[i][0]
        assert np.array_equal(probs[i].state(probs[i].N).cpu().numpy(), batched[i][1][-1])


@pytest.mark.parametrize("coarse", ["fp64", "delta32"])
def test_batch_with_sources_both_coarse_forms_bitwise(ps, coarse):
    """Batches of problems with time-dependent sources, in the FP64 coarse form and the FP32
    increment form: the batched run equals each problem's own run bitwise (iteration counts,
    histories, states); one problem against the oracle within the FP32 bound."""
    cfgs = wl.batch256(count=6, seed=13, sizes=(31, 47, 64), slices=(4, 8, 16), s_range=(3, 12))
    rng = np.random.default_rng(14)
    probs, u0s, srcs = [], [], []
    for c in cfgs:
        nx, ny = c["n"]
        src = rng.standard_normal((ny, nx))
        src_t = 1.0 + 0.5 * np.sin(0.4 * np.arange(c["N"] * c["s"] + 1))
        grid = ps.Grid(c["n"])
        op = ps.Operator(grid, a=dev(c["a"]), src=dev(src), src_t=src_t)
        sp = ps.Splitting(op)
        p = ps.Problem(sp, c["T"], c["N"], 1, c["s"], precision="mixed", coarse_mode=coarse)
        p._keep = (grid, op, sp)
        probs.append(p)
        u0s.append(dev(c["u0"]))
        srcs.append((src, src_t))
    ref = []
    for p, u in zip(probs, u0s):
        k = p.run(u, 1e-8)
        ref.append((k, p.history(), snapshot(p)))
    batch = ps.Batch(probs)
    its = batch.run(u0s, 1e-8)
    assert its == [r[0] for r in ref]
    for i, p in enumerate(probs):
        assert np.array_equal(p.history(), ref[i][1]), i
        got = snapshot(p)
        for n in range(p.N + 1):
            assert np.array_equal(got[n], ref[i][2][n]), (i, n)
    c = cfgs[0]
    orp = orc.Problem(c["n"], a=c["a"], src=srcs[0][0], src_t=srcs[0][1])
    U_ref, _, _ = orc.parareal(orp, c["T"], c["N"], 1, c["s"], c["u0"], 1e-8)
    err = np.abs(ref[0][2][-1] - U_ref[-1]).max() / np.abs(U_ref[-1]).max()
    assert err < 4.0 * c["s"] * c["N"] * 2 * 2.0 ** -24


@pytest.mark.parametrize("coarse", ["fp64", "delta32"])
def test_3d_batch_equals_individual_runs_bitwise(ps, coarse):
    """Batches of 3-D problems (three fine tile directions, coarse x rows over y and z, y- and
    z-line sweeps with the epilogue on z): every state, history and iteration count equal the
    problems' own runs bitwise, for both coarse forms, with a source on some problems."""
    rng = np.random.default_rng(91)
    shapes = [(17, 13, 11), (23, 9, 15), (31, 17, 9), (12, 20, 7)]
    probs, u0s = [], []
    for i, n in enumerate(shapes):
        a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
        src = rng.standard_normal(n[::-1]) if i % 2 == 0 else None
        N, s = (4, 8)[i % 2], 3 + i
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), src=None if src is None else dev(src))
        sp = ps.Splitting(op)
        prob = ps.Problem(sp, 0.4, N, 1, s, precision="mixed", coarse_mode=coarse)
        prob._keep = (grid, op, sp)
        probs.append(prob)
        u0s.append(dev(rng.standard_normal(n[::-1])))
    ref = []
    for p, u in zip(probs, u0s):
        it = p.run(u, 1e-9)
        ref.append((it, snapshot(p), p.history()))
    batch = ps.Batch(probs)
    for _ in range(2):
        its = batch.run(u0s, 1e-9)
        assert its == [r[0] for r in ref]
        for p, (it, st, h) in zip(probs, ref):
            got = snapshot(p)
            for n in range(p.N + 1):
                assert np.array_equal(got[n], st[n]), n
            assert np.array_equal(p.history(), h)
    # mixed dimensions are refused
    g2 = ps.Grid((9, 8))
    op2 = ps.Operator(g2)
    p2 = ps.Problem(ps.Splitting(op2), 0.4, 4, 1, 3, precision="mixed", coarse_mode=coarse)
    with pytest.raises(ps.PsError):
        batch.add(p2)


@pytest.mark.parametrize("coarse", ["fp64", "delta32"])
def test_batch_tile_shapes_of_mixed_line_lengths_bitwise(ps, coarse):
    """A batch whose lines range from 9 to 511 nodes: every tile of the grouped launch reserves
    the largest tile (511-node x lines with a source), so the batch gives the shorter lines more
    positions per tile (two for 255 nodes, four for 127 and fewer), with ragged last tiles
    (21, 127, 255 and 17 positions).  States, histories and iteration counts equal each
    problem's own run (one position per tile) bitwise."""
    rng = np.random.default_rng(93)
    shapes = [(511, 9), (255, 21), (63, 127), (17, 255)]
    probs, u0s = [], []
    for i, n in enumerate(shapes):
        a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
        src = rng.standard_normal(n[::-1]) if i % 2 == 0 else None
        N, s = (4, 8)[i % 2], 3 + i
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), src=None if src is None else dev(src))
        sp = ps.Splitting(op)
        prob = ps.Problem(sp, 0.4, N, 1, s, precision="mixed", coarse_mode=coarse, tile_positions=1)
        prob._keep = (grid, op, sp)
        probs.append(prob)
        u0s.append(dev(rng.standard_normal(n[::-1])))
    ref = []
    for p, u in zip(probs, u0s):
        it = p.run(u, 1e-9)
        ref.append((it, snapshot(p), p.history()))
    batch = ps.Batch(probs)
    for _ in range(2):
        its = batch.run(u0s, 1e-9)
        assert its == [r[0] for r in ref]
        for p, (it, st, h) in zip(probs, ref):
            got = snapshot(p)
            for n in range(p.N + 1):
                assert np.array_equal(got[n], st[n]), n
            assert np.array_equal(p.history(), h)
