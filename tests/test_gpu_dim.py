"""GPU parity of the dimensional-splitting path against the FP64 CPU oracle.

Every call goes through the C ABI (libps.so) via the thin binding.  FP64 results
must match the oracle to 1e-12 in relative max-norm with equal parareal
iteration counts; the FP32 line-solve form must stay within the bound stated in
``mixed_bound`` (C * s * N * M * 2^-24 relative, C = 4).
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def make(ps, n, a=None, c=0.0, src=None, src_t=None, T=1.0, N=4, g=1, s=4, precision="fp64", split="dim",
         boxes=(1, 1), overlap=0.0):
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=None if a is None else dev(a), c=c, src=None if src is None else dev(src), src_t=src_t)
    sp = ps.Splitting(op, split, boxes, overlap)
    prob = ps.Problem(sp, T, N, g, s, precision=precision)
    prob._keep = (grid, op, sp)
    orp = orc.Problem(n, a=a, c=c, src=src, src_t=src_t, split=split, boxes=boxes, overlap=overlap)
    return prob, orp


def mixed_bound(s, N, M):
    return 4.0 * s * N * M * 2.0 ** -24


SIZES = [(1, 1), (2, 3), (7, 5), (33, 31), (64, 17), (5, 4, 3), (17, 9, 12), (1, 6, 2)]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("variable", [False, True])
def test_substep_solve_matches_oracle(ps, n, variable):
    rng = np.random.default_rng(hash((n, variable)) % 2 ** 32)
    a = np.exp(0.5 * rng.standard_normal([v + 2 for v in reversed(n)])) if variable else None
    prob, orp = make(ps, n, a=a, c=0.3, T=0.7, N=3, g=1, s=5)
    b = rng.standard_normal(n[::-1])
    for which, tau in ((0, 0.7 / 3 / 5), (1, 0.7 / 3)):
        for m in range(len(n)):
            x = dev(b)
            prob.substep_solve(which, m, x)
            ref = orc.substep_solve(orp, m, tau, b)
            assert relmax(x.cpu().numpy(), ref) < RTOL64, (which, m)


@pytest.mark.parametrize("n", [(9, 8), (6, 5, 7), (255, 3)])
def test_propagate_with_source_matches_oracle(ps, n):
    rng = np.random.default_rng(7)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    N, s = 3, 4
    src = rng.standard_normal(n[::-1])
    src_t = np.cos(0.3 * np.arange(N * s + 1))
    prob, orp = make(ps, n, a=a, c=0.1, src=src, src_t=src_t, T=0.5, N=N, g=2, s=s)
    u = rng.standard_normal(n[::-1])
    x = dev(u)
    prob.propagate(0, 5, x, t0=2, tstride=1)
    ref = orc.propagate(orp, 0.5 / N / s, 5, u, t0=2, tstride=1)
    assert relmax(x.cpu().numpy(), ref) < RTOL64
    x = dev(u)
    prob.propagate(1, 2, x, t0=0, tstride=2)
    ref = orc.propagate(orp, 0.5 / N / 2, 2, u, t0=0, tstride=2)
    assert relmax(x.cpu().numpy(), ref) < RTOL64


def test_parareal_heat2d_63_full_size(ps):
    """63x63, N = 16, s = 64, tol 1e-10: equal iteration count, states within 1e-12."""
    cfg = wl.heat2d_63()
    prob, orp = make(ps, cfg["n"], T=cfg["T"], N=cfg["N"], g=1, s=cfg["s"])
    it = prob.run(dev(cfg["u0"]), cfg["tol"])
    U_ref, h_ref, it_ref = orc.parareal(orp, cfg["T"], cfg["N"], 1, cfg["s"], cfg["u0"], cfg["tol"])
    assert it == it_ref == 12
    hist = prob.history()
    np.testing.assert_allclose(hist, h_ref, rtol=1e-6, atol=1e-14)
    for n in range(cfg["N"] + 1):
        assert relmax(prob.state(n).cpu().numpy(), U_ref[n]) < RTOL64, n


@pytest.mark.parametrize("n,N,s,g", [((15, 13, 11), 6, 8, 1), ((31, 29), 8, 16, 2), ((20, 9, 6), 5, 6, 3)])
def test_parareal_variable_coefficient_source(ps, n, N, s, g):
    rng = np.random.default_rng(11)
    a = np.exp(0.4 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    src_t = 1.0 + np.sin(np.arange(N * s + 1) * 0.2)
    prob, orp = make(ps, n, a=a, c=0.5, src=src, src_t=src_t, T=0.4, N=N, g=g, s=s)
    u0 = rng.standard_normal(n[::-1])
    tol = 1e-9
    it = prob.run(dev(u0), tol)
    U_ref, h_ref, it_ref = orc.parareal(orp, 0.4, N, g, s, u0, tol)
    assert it == it_ref
    for j in range(N + 1):
        assert relmax(prob.state(j).cpu().numpy(), U_ref[j]) < RTOL64, j


def test_finite_termination_bitwise_on_gpu(ps):
    """U_n^k equals the GPU's own sequential fine solution bitwise for n <= k (Sec. 3)."""
    rng = np.random.default_rng(12)
    n, N, s = (21, 19), 6, 5
    a = np.exp(0.4 * rng.standard_normal((n[1] + 2, n[0] + 2)))
    prob, _ = make(ps, n, a=a, src=rng.standard_normal(n[::-1]), T=0.3, N=N, g=1, s=s)
    u0 = dev(rng.standard_normal(n[::-1]))
    fine = prob.fine_sequential(u0).cpu().numpy()
    for k in range(1, N + 1):
        it = prob.run(u0, 0.0, max_iter=k)
        assert it == k
        for j in range(k + 1):
            assert np.array_equal(prob.state(j).cpu().numpy(), fine[j]), (k, j)


def test_coarse_sequential_matches_oracle(ps):
    cfg = wl.heat3d_255(n=15, N=4, s=6)
    prob, orp = make(ps, cfg["n"], a=cfg["a"], src=cfg["src"], T=1.0, N=4, g=1, s=6)
    U = prob.coarse_sequential(dev(cfg["u0"])).cpu().numpy()
    ref = orc.coarse_sequential(orp, 1.0, 4, 1, 6, cfg["u0"])
    assert relmax(U, ref) < RTOL64


@pytest.mark.parametrize("n,N,s", [((33, 31), 8, 16), ((15, 14, 13), 6, 8)])
def test_mixed_precision_within_stated_bound(ps, n, N, s):
    """FP32 line solves in F; result vs the FP64 oracle within C s N M 2^-24 (C = 4)."""
    rng = np.random.default_rng(13)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    prob, orp = make(ps, n, a=a, src=src, T=1.0, N=N, g=1, s=s, precision="mixed")
    u0 = rng.standard_normal(n[::-1])
    it = prob.run(dev(u0), 1e-8)
    U_ref, _, it_ref = orc.parareal(orp, 1.0, N, 1, s, u0, 1e-8)
    assert abs(it - it_ref) <= 1
    err = relmax(prob.state(N).cpu().numpy(), U_ref[N])
    assert err < mixed_bound(s, N, len(n)), err
    # the mixed fixed point is the mixed fine solution: k = N reproduces it bitwise
    u0d = dev(u0)
    fine = prob.fine_sequential(u0d).cpu().numpy()
    prob.run(u0d, 0.0, max_iter=N)
    assert np.array_equal(prob.state(N).cpu().numpy(), fine[N])


def test_host_entry_point_matches_device_entry_point(ps):
    cfg = wl.heat2d_63(n=31, N=8, s=16)
    prob, _ = make(ps, cfg["n"], T=1.0, N=8, g=1, s=16)
    it = prob.run(dev(cfg["u0"]), 1e-10)
    ref = prob.state(8).cpu().numpy()
    u0h = torch.as_tensor(cfg["u0"]).contiguous().pin_memory()
    uNh = torch.empty_like(u0h).pin_memory()
    it2 = prob.run_host(u0h, uNh, 1e-10)
    assert it == it2 and np.array_equal(uNh.numpy(), ref)


def test_invalid_arguments_are_rejected(ps):
    grid = ps.Grid((5, 5))
    op = ps.Operator(grid)
    sp = ps.Splitting(op)
    with pytest.raises(ps.PsError) as e:
        ps.Problem(sp, 1.0, 4, 3, 8)  # f_steps % g_steps != 0
    assert e.value.code == 1
    with pytest.raises(ps.PsError):
        ps.Problem(sp, -1.0, 4, 1, 8)
    with pytest.raises(ps.PsError) as e:
        ps.Problem(sp, 1.0, 4, 1, 8, schedule=7)
    assert e.value.code == 1
    prob = ps.Problem(sp, 1.0, 4, 1, 8)
    with pytest.raises(ps.PsError):
        prob.state(5)
    with pytest.raises(ValueError):
        prob.run(torch.zeros(3, dtype=torch.float64, device="cuda"), 1e-8)


def test_nonfinite_input_is_reported(ps):
    prob, _ = make(ps, (9, 9), N=4, s=4)
    u0 = np.ones((9, 9))
    u0[3, 3] = np.nan
    with pytest.raises(ps.PsError) as e:
        prob.run(dev(u0), 1e-8)
    assert e.value.code == 4


@pytest.mark.parametrize("n", [(511, 9), (7, 300), (6, 5, 300), (300, 4, 3)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fine_sequential_long_lines_chunked_tiles(ps, n, precision):
    """Lines longer than one TMA box (256 nodes) are moved in several chunks."""
    rng = np.random.default_rng(17)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    N, s = 3, 2
    src_t = 1.0 + np.cos(np.arange(N * s + 1))
    prob, orp = make(ps, n, a=a, c=0.2, src=src, src_t=src_t, T=0.01, N=N, g=1, s=s, precision=precision)
    u0 = rng.standard_normal(n[::-1])
    got = prob.fine_sequential(dev(u0)).cpu().numpy()
    ref = orc.fine_sequential(orp, 0.01, N, s, u0)
    bound = RTOL64 if precision == "fp64" else mixed_bound(s, N, len(n))
    for j in range(N + 1):
        assert relmax(got[j], ref[j]) < bound, j


def test_fine_sequential_on_recycled_device_memory(ps):
    """Device memory that cudaMalloc hands back keeps its old contents: fill memory with
    all-ones words, release it, then create a problem (its status flags are carved from the
    same pool) and check that the fine propagator still runs every sweep."""
    junk = torch.full((1 << 26,), -1, dtype=torch.int32, device="cuda")
    del junk
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    rng = np.random.default_rng(19)
    n, N, s = (7, 300), 3, 2
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    prob, orp = make(ps, n, a=a, T=0.01, N=N, g=1, s=s)
    u0 = rng.standard_normal(n[::-1])
    got = prob.fine_sequential(dev(u0)).cpu().numpy()
    ref = orc.fine_sequential(orp, 0.01, N, s, u0)
    for j in range(N + 1):
        assert relmax(got[j], ref[j]) < RTOL64, j


def make_delta(ps, n, a=None, src=None, T=1.0, N=4, s=4):
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=None if a is None else dev(a), src=None if src is None else dev(src))
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, T, N, 1, s, precision="mixed", coarse_mode="delta32")
    prob._keep = (grid, op, sp)
    return prob, orc.Problem(n, a=a, src=src)


@pytest.mark.parametrize("n,N,s,variable", [((33, 31), 8, 16, True), ((15, 14, 13), 6, 8, True), ((63, 63), 16, 64, False),
                                             ((300, 11), 5, 4, True)])
def test_coarse_increment_form_fp32(ps, n, N, s, variable):
    """Coarse increment form (FP32 line solves on U_n^k - U_n^{k-1}, FP64 correction and test) with
    FP32 fine solves: U_N within the FP32 bound of the FP64 oracle, iteration count within one of
    the oracle's, finite termination bitwise, and k = N reproduces the FP32 fine solution."""
    rng = np.random.default_rng(23)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)])) if variable else None
    src = rng.standard_normal(n[::-1])
    prob, orp = make_delta(ps, n, a=a, src=src, T=1.0, N=N, s=s)
    u0 = rng.standard_normal(n[::-1])
    tol = 1e-8
    it = prob.run(dev(u0), tol)
    U_ref, _, it_ref = orc.parareal(orp, 1.0, N, 1, s, u0, tol)
    assert abs(it - it_ref) <= 1, (it, it_ref)
    err = relmax(prob.state(N).cpu().numpy(), U_ref[N])
    assert err < mixed_bound(s, N, len(n)), err
    u0d = dev(u0)
    fine = prob.fine_sequential(u0d).cpu().numpy()
    for k in (1, 2, N):
        assert prob.run(u0d, 0.0, max_iter=k) == k
        for j in range(k + 1):
            assert np.array_equal(prob.state(j).cpu().numpy(), fine[j]), (k, j)


def test_coarse_increment_form_is_rejected_where_unsupported(ps):
    prob, _ = make_delta(ps, (17, 15), a=np.ones((17, 19)), N=4, s=4)
    u0 = dev(np.ones((15, 17)))
    prob.run(u0, 1e-8)
    with pytest.raises(ps.PsError) as e:
        prob.vjp(prob.state(4), 1e-8)
    assert e.value.code == 6
    # a batch takes increment-form problems, but not mixed with FP64-coarse ones
    other, _ = make_delta(ps, (17, 15), a=np.ones((17, 19)), N=4, s=4)
    ps.Batch([prob, other])
    grid = ps.Grid((17, 15))
    op = ps.Operator(grid, a=dev(np.ones((17, 19))))
    fp64_coarse = ps.Problem(ps.Splitting(op), 1.0, 4, 1, 4, precision="mixed")
    with pytest.raises(ps.PsError) as e:
        ps.Batch([prob, fp64_coarse])
    assert e.value.code == 1
    # the sequential coarse solution keeps the FP64 coarse steps
    ref = orc.coarse_sequential(orc.Problem((17, 15), a=np.ones((17, 19))), 1.0, 4, 1, 4, np.ones((15, 17)))
    assert relmax(prob.coarse_sequential(u0).cpu().numpy(), ref) < RTOL64


@pytest.mark.parametrize("n,positions", [((40, 37, 33), 1), ((64, 17), 2), ((300, 11), 1)])
def test_fp32_tiles_one_line_per_thread(ps, n, positions):
    """FP32 tiles solved with one line per thread (twice the threads per tile) give the same
    states as two lines per thread, bitwise: each line's recurrence is the same arithmetic."""
    rng = np.random.default_rng(29)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    u0 = dev(rng.standard_normal(n[::-1]))
    out = []
    for vec in (2, 1):
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), src=dev(src))
        sp = ps.Splitting(op)
        prob = ps.Problem(sp, 0.5, 6, 1, 5, precision="mixed", tile_positions=positions, tile_lines_per_thread=vec)
        prob.run(u0, 1e-8)
        out.append([prob.state(j).cpu().numpy() for j in range(7)])
    for j in range(7):
        assert np.array_equal(out[0][j], out[1][j]), j
    U_ref, _, _ = orc.parareal(orc.Problem(n, a=a, src=src), 0.5, 6, 1, 5, u0.cpu().numpy(), 1e-8)
    assert relmax(out[1][6], U_ref[6]) < mixed_bound(5, 6, len(n))


@pytest.mark.parametrize("n", [(63, 63), (255, 9, 7), (40, 37, 33)])
def test_coarse_x_schedules_thomas_pcr_hybrid(ps, n):
    """The FP32 increment form's coarse x-sweep in its three schedules (Thomas per row, PCR per
    warp, hybrid segmented scans per warp): the same iteration count and states within the FP32
    rounding of the coarse increment of each other, and within the FP32 bound of the oracle."""
    rng = np.random.default_rng(71)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    u0 = dev(rng.standard_normal(n[::-1]))
    N, s, T = 8, 6, 0.4
    out = {}
    for sched in (ps.PS_SCHED_THOMAS, ps.PS_SCHED_PCR, ps.PS_SCHED_HYBRID):
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), src=dev(src))
        sp = ps.Splitting(op)
        prob = ps.Problem(sp, T, N, 1, s, precision="mixed", coarse_mode="delta32", schedule=sched)
        it = prob.run(u0, 1e-10)
        out[sched] = (it, [prob.state(j).cpu().numpy() for j in range(N + 1)])
    its = {v[0] for v in out.values()}
    assert len(its) == 1, its
    ref = out[ps.PS_SCHED_HYBRID][1]
    # the coarse propagator only steers the iteration: at convergence every schedule sits within
    # the increment tolerance of the same FP32-fine fixed point
    for sched in (ps.PS_SCHED_THOMAS, ps.PS_SCHED_PCR):
        for j in range(N + 1):
            assert relmax(out[sched][1][j], ref[j]) < 1e-8, (sched, j)
    U_ref, _, _ = orc.parareal(orc.Problem(n, a=a, src=src), T, N, 1, s, u0.cpu().numpy(), 1e-10)
    assert relmax(out[ps.PS_SCHED_PCR][1][N], U_ref[N]) < mixed_bound(s, N, len(n))


def test_autotune_record_lists_every_schedule(ps):
    n = (127, 63, 31)
    rng = np.random.default_rng(72)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=dev(a))
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, 0.5, 32, 1, 4, precision="mixed", coarse_mode="delta32")
    u0 = dev(rng.standard_normal(n[::-1]))
    prob.run(u0, 1e-8)
    before = prob.state(32).cpu().numpy()
    choice = prob.autotune(budget_ms=40)
    rec = prob.autotune_record()
    names = [r[0] for r in rec]
    assert {"coarse-x32:thomas", "coarse-x32:pcr", "coarse-x32:hybrid", "coarse:staged", "coarse:streamed"} <= set(names)
    assert not any(nm.startswith("coarse-corr:") for nm in names)  # the increment form fuses its epilogue
    assert any(nm.startswith("fine:") for nm in names)
    for group in ("fine:", "coarse-x32:", "coarse:"):
        chosen = [r for r in rec if r[0].startswith(group) and r[2]]
        assert len(chosen) == 1, (group, rec)
        assert chosen[0][1] == min(r[1] for r in rec if r[0].startswith(group))
    assert choice // 100000 in (1, 2)
    prob.run(u0, 1e-8)
    assert relmax(prob.state(32).cpu().numpy(), before) < 1e-7


@pytest.mark.parametrize("prec,coarse,N", [("mixed", "fp64", 70), ("mixed", "delta32", 64), ("fp64", "fp64", 40)])
def test_fine_phase_beside_chain_is_bitwise_serial(ps, prec, coarse, N):
    """The fine phase run slot group by slot group on a side stream, with the coarse chain
    following each group, computes exactly what the serial order computes: every state and the
    history bitwise equal, for runs ending at convergence and at k = N."""
    n = (31, 27, 23)
    rng = np.random.default_rng(73)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    u0 = dev(rng.standard_normal(n[::-1]))
    res = []
    for overlap in (True, False):
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), src=dev(src))
        sp = ps.Splitting(op)
        prob = ps.Problem(sp, 0.5, N, 1, 4, precision=prec, coarse_mode=coarse, overlap_phases=overlap)
        out = []
        for tol, mi in ((1e-9, 0), (0.0, 5)):
            it = prob.run(u0, tol, mi)
            out.append((it, prob.history(), [prob.state(j).cpu().numpy() for j in range(N + 1)]))
        res.append(out)
    for (it1, h1, s1), (it2, h2, s2) in zip(res[0], res[1]):
        assert it1 == it2 and np.array_equal(h1, h2)
        for j in range(N + 1):
            assert np.array_equal(s1[j], s2[j]), j


@pytest.mark.parametrize("n", [(33, 31), (255, 9, 7), (40, 37, 33), (300, 130), (64, 5, 70)])
def test_fp64_coarse_chunked_sweeps_equal_staged_bitwise(ps, n):
    """The streamed FP64 coarse sweeps pass each line through shared memory in chunks (x: 16
    nodes of 128 rows per CTA; y, z: per-thread asynchronous copies one chunk ahead); the staged
    sweeps hold whole lines.  Both run the same operations in the same order, so an FP64 run
    gives the same bits either way (history, iteration count, every state), and matches the
    oracle to 1e-12.  Shapes: ragged chunks, rows of a CTA crossing grid planes, a partial last
    CTA, long rows and long z-lines."""
    rng = np.random.default_rng(74)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    src_t = 1.0 + 0.2 * np.cos(np.arange(6 * 4 + 1))
    u0 = rng.standard_normal(n[::-1])
    N, s, T = 6, 4, 0.4
    out = {}
    for cs in ("staged", "streamed"):
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), c=0.2, src=dev(src), src_t=src_t)
        sp = ps.Splitting(op)
        prob = ps.Problem(sp, T, N, 1, s, coarse_sweep=cs)
        it = prob.run(dev(u0), 1e-10)
        out[cs] = (it, prob.history(), [prob.state(j).cpu().numpy() for j in range(N + 1)])
        prob.run(dev(u0), 0.0, 2)
        out[cs + "2"] = [prob.state(j).cpu().numpy() for j in range(N + 1)]
    assert out["staged"][0] == out["streamed"][0]
    assert np.array_equal(out["staged"][1], out["streamed"][1])
    for j in range(N + 1):
        assert np.array_equal(out["staged"][2][j], out["streamed"][2][j]), j
        assert np.array_equal(out["staged2"][j], out["streamed2"][j]), j
    U_ref, _, it_ref = orc.parareal(orc.Problem(n, a=a, c=0.2, src=src, src_t=src_t), T, N, 1, s, u0, 1e-10)
    assert out["streamed"][0] == it_ref
    for j in range(N + 1):
        assert relmax(out["streamed"][2][j], U_ref[j]) < RTOL64, j


@pytest.mark.parametrize("n,prec", [((255, 9, 140), "mixed"), ((200, 150), "mixed"), ((200, 150), "fp64")])
def test_16_slot_tiles_are_bitwise_the_32_slot_tiles(ps, n, prec):
    """Tiles of 16 slots (64-byte FP32 rows, one TMA box per tile) compute exactly what the
    default 32-slot tiles compute: same history, same states; and match the oracle within the
    FP32 bound (or 1e-12 in FP64)."""
    rng = np.random.default_rng(75)
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    src = rng.standard_normal(n[::-1])
    u0 = dev(rng.standard_normal(n[::-1]))
    N, s, T = 6, 4, 0.3
    out = {}
    # (pipeline, slots per tile): one-shot 32-slot tiles and 16-slot tiles (64-byte FP32 rows)
    for key in ((2, 0), (2, 16)):
        grid = ps.Grid(n)
        op = ps.Operator(grid, a=dev(a), src=dev(src))
        sp = ps.Splitting(op)
        prob = ps.Problem(sp, T, N, 1, s, precision=prec, tile_positions=1, tile_pipeline=key[0], tile_slots=key[1])
        it = prob.run(u0, 1e-9)
        out[key] = (it, prob.history(), [prob.state(j).cpu().numpy() for j in range(N + 1)])
    for key in ((2, 16),):
        assert out[(2, 0)][0] == out[key][0] and np.array_equal(out[(2, 0)][1], out[key][1]), key
        for j in range(N + 1):
            assert np.array_equal(out[(2, 0)][2][j], out[key][2][j]), (key, j)
    out[3] = out[(2, 16)]
    U_ref, _, _ = orc.parareal(orc.Problem(n, a=a, src=src), T, N, 1, s, u0.cpu().numpy(), 1e-9)
    bar = mixed_bound(s, N, len(n)) if prec == "mixed" else RTOL64
    assert relmax(out[3][2][N], U_ref[N]) < bar
