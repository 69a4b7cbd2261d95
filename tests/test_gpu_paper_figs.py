"""Sec. 5.1, Figs. 4-6, with the dimensional splitting at the paper's h = 1e-3, on the GPU.

The manufactured problem u = sin(2 pi t) sin(2 pi x) sin(2 pi y) (eq. heat_prob, D = I), 999^2
interior nodes, T = 1, Delta T = 0.05 (N = 20), u0 = 0.  Errors of the k-th parareal iterate
against the fine solution (max over the coarse times of the h-weighted 2-norm, Sec. 5):

  - Parareal/FIE-FIE decays geometrically, and the more fine steps per slice, the slower
    (Fig. 5's statement for FIE-FIE): the contraction per iteration grows with s.
  - Parareal/FIE-DR decays geometrically too; s = 2 is its slowest case (Theorem 2: at small s
    the FIE-DR factor stays near 1 over a wider range of eigenvalues, Fig. 5(b)).
  - The iteration counts to 1e-6 are robust in h (Fig. 6(b)): within one of each other for
    h = 1/100 .. 1/1000, for both methods.

The measured rows are recorded next to the test log (PS_TEST_RECORD).  The paper also reports a
change of slope of FIE-DR at the 10th iteration (Fig. 4, s = 20); on this grid the FIE-DR
error keeps contracting by ~0.1 per iteration until it meets the rounding floor near the 12th
iteration, so that statement is not asserted.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2502_08370_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
T, N = 1.0, 20


@pytest.fixture(scope="module")
def ps():
    from paper_2502_08370_gb300 import build
    build.build()
    import paper_2502_08370_gb300 as ps
    return ps


def make(ps, n, s, fine):
    S, st, _ = wl.manufactured((n, n), T, N, s)
    grid = ps.Grid((n, n))
    op = ps.Operator(grid, src=torch.as_tensor(S).cuda(), src_t=st)
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, T, N, 1, s, fine_method=fine)
    prob._keep = (grid, op, sp)
    return prob


def errors_vs_fine(ps, n, s, fine, kmax):
    prob = make(ps, n, s, fine)
    u0 = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    F = prob.fine_sequential(u0)
    h = 1.0 / (n + 1)
    out = []
    for k in range(1, kmax + 1):
        assert prob.run(u0, 0.0, max_iter=k) == k
        out.append(max(float(torch.sqrt(h * h * ((prob.state(j) - F[j]) ** 2).sum())) for j in range(1, N + 1)))
    return np.array(out)


def record(name, data):
    path = os.environ.get("PS_TEST_RECORD")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, **data}) + "\n")


def mean_ratio(e):
    # contraction per iteration over the first iterations (well above the rounding floor)
    return float(np.exp(np.mean(np.log(e[1:7] / e[0:6]))))


def test_fig45_contraction_against_s_at_h_1e3(ps):
    rows = {}
    for fine, ss in (("fie", (2, 5, 20)), ("dr", (2, 5, 20))):
        for s in ss:
            e = errors_vs_fine(ps, 999, s, fine, 8)
            rows[f"{fine}_s{s}"] = e.tolist()
            # geometric decay: every step contracts
            assert np.all(e[1:] < 0.5 * e[:-1]), (fine, s, e)
    record("fig45_dim_h1e-3", {"err_vs_fine": rows})
    q = {k: mean_ratio(np.array(v)) for k, v in rows.items()}
    # FIE-FIE: slower for more fine steps per slice
    assert q["fie_s2"] < q["fie_s5"] < q["fie_s20"] < 0.2, q
    # FIE-DR: s = 2 is the slowest of its cases
    assert q["dr_s2"] > q["dr_s5"] and q["dr_s2"] > q["dr_s20"], q


def test_fig6b_iterations_robust_in_h(ps):
    counts = {}
    for fine in ("fie", "dr"):
        for n in (99, 199, 499, 999):
            prob = make(ps, n, 20, fine)
            counts[f"{fine}_n{n}"] = prob.run(torch.zeros((n, n), dtype=torch.float64, device="cuda"), 1e-6)
    record("fig6b_dim_iterations_to_1e-6", {"iterations": counts})
    for fine in ("fie", "dr"):
        its = [counts[f"{fine}_n{n}"] for n in (99, 199, 499, 999)]
        assert max(its) - min(its) <= 1, (fine, its)
