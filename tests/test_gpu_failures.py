"""Failure paths on the GPU without a GPU fault: the device-side wait limit runs out on a
barrier that nothing arrives at, the host reads PS_ERR_DEVICE_TIMEOUT, and the context stays
usable; invalid and non-finite inputs are reported with their status codes."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    from paper_2502_08370_gb300 import build
    build.build()
    import paper_2502_08370_gb300 as ps
    return ps


def test_wait_limit_reports_timeout_and_context_survives(ps):
    t0 = time.perf_counter()
    rc = ps.selftest_wait_timeout(20000)
    dt = time.perf_counter() - t0
    assert rc == 5, ps.lib().ps_last_error()
    assert b"bounded wait" in ps.lib().ps_last_error()
    assert dt >= 0.02
    # the context is intact: a parareal run right after matches the oracle
    n, N, s = (21, 18), 4, 6
    rng = np.random.default_rng(31)
    u0 = rng.standard_normal(n[::-1])
    grid = ps.Grid(n)
    op = ps.Operator(grid)
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, 0.5, N, 1, s)
    it = prob.run(torch.as_tensor(u0).cuda(), 1e-10)
    U_ref, _, it_ref = orc.parareal(orc.Problem(n), 0.5, N, 1, s, u0, 1e-10)
    assert it == it_ref
    ref = U_ref[N]
    assert np.abs(prob.state(N).cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    # a second timeout in a row behaves the same
    assert ps.selftest_wait_timeout(1000) == 5
