"""The no-allocation coarse solve gives the allocating coarse solve's results.

ps_run_coarse_sequential_noalloc serves callers that cannot allocate device memory at
call time (for example code running inside a host callback or an allocator hook, where
cudaMalloc is not allowed).  It keeps its working state in a fixed per-device array of
PS_NOALLOC_MAX_UNKNOWNS doubles instead.  This file is collected last so that a run that
stops at the first failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def make(ps, n, a=None, src=None, src_t=None, N=6, g=1, s=4, split="dim", boxes=(1, 1), overlap=0.0):
    grid = ps.Grid(n)
    op = ps.Operator(grid, a=None if a is None else dev(a), src=None if src is None else dev(src), src_t=src_t)
    sp = ps.Splitting(op, split, boxes, overlap)
    prob = ps.Problem(sp, 0.5, N, g, s)
    prob._keep = (grid, op, sp)
    return prob


def noalloc_call(ps, prob, u0, out):
    """Direct C-ABI call of the no-allocation entry point."""
    lib = ps.lib()
    rc = lib.ps_run_coarse_sequential_noalloc(prob._h, ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_uint64(torch.cuda.current_stream().cuda_stream))
    return rc


CASES = [
    ("dim2d", dict(n=(63, 47))),
    ("dim3d", dict(n=(17, 15, 13), g=2)),
    ("dd2d", dict(n=(41, 37), split="dd", boxes=(4, 3), overlap=4 / 42.0)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_coarse_solve_twice(ps, name, kw):
    rng = np.random.default_rng(31)
    n = kw["n"]
    a = np.exp(0.3 * rng.standard_normal([v + 2 for v in reversed(n)]))
    N, s = 6, 4
    src = rng.standard_normal(n[::-1])
    src_t = np.cos(0.2 * np.arange(N * s + 1))
    prob = make(ps, n, a=a, src=src, src_t=src_t, N=N, s=s, g=kw.get("g", 1), split=kw.get("split", "dim"),
                boxes=kw.get("boxes", (1, 1)), overlap=kw.get("overlap", 0.0))
    u0 = dev(rng.standard_normal(n[::-1]))
    ref = prob.coarse_sequential(u0).cpu().numpy()
    for call in range(2):  # the shared scratch keeps the previous call's contents
        out = torch.full((N + 1,) + tuple(n[::-1]), float("nan"), dtype=torch.float64, device="cuda")
        rc = noalloc_call(ps, prob, u0, out)
        assert rc == 0, ps.lib().ps_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= RTOL64, (call, err)


def test_noalloc_rejects_grids_beyond_its_limit(ps):
    n = (1025, 1025)  # 1,050,625 unknowns > 2^20
    assert n[0] * n[1] > ps.PS_NOALLOC_MAX_UNKNOWNS
    prob = make(ps, n, N=1, s=1)
    u0 = torch.zeros(n[::-1], dtype=torch.float64, device="cuda")
    out = torch.zeros((2,) + n[::-1], dtype=torch.float64, device="cuda")
    rc = noalloc_call(ps, prob, u0, out)
    assert rc == 1
    assert b"at most" in ps.lib().ps_last_error()


def test_noalloc_full_workload_slice(ps):
    """The heat2d workload (63^2, N = 16) through the binding's method."""
    cfg = wl.heat2d_63()
    prob = make(ps, cfg["n"], N=cfg["N"], s=cfg["s"])
    u0 = dev(cfg["u0"])
    ref = prob.coarse_sequential(u0).cpu().numpy()
    out = torch.empty((cfg["N"] + 1,) + tuple(cfg["n"][::-1]), dtype=torch.float64, device="cuda")
    got = prob.coarse_sequential_noalloc(u0, out).cpu().numpy()
    assert np.abs(got - ref).max() <= RTOL64 * np.abs(ref).max()
