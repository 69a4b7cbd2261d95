"""The paper's printed errors (Sec. 5.1, scalability experiment) as pins of the oracle.

The fine approximation's error is reproduced to every printed digit; it does
not depend on the overlap ramp, which the paper leaves unspecified.  The
coarse errors do depend on it: for q = 2 and 4 they agree within a few
percent, for q = 8 only in order of magnitude; the parareal errors after five
iterations agree in order of magnitude.
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
from paper_2502_08370_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_scalability_errors.json")))
n, T, N, s = 99, 1.0, 32, 100  # h = 0.01, DeltaT = 1/32, delta t = 1/3200


def setup():
    S, st, exact = wl.manufactured((n, n), T, N, s)
    h = 1.0 / (n + 1)

    def err(U):
        return max(np.sqrt(h * h * np.sum((U[j] - exact(j * T / N)) ** 2)) for j in range(1, N + 1))

    def strips(q, beta):
        return orc.Problem((n, n), src=S, src_t=st, split="dd", boxes=(2 * q, 1), overlap=beta)

    return err, strips


def test_fine_error_matches_printed_value():
    err, strips = setup()
    U = orc.fine_sequential(strips(2, 1 / 16), T, N, s, np.zeros((n, n)))
    e = err(U)
    assert abs(e - GOLD["printed"]["fine_error"]) <= 0.5e-7, e  # 5 significant digits


def test_coarse_errors_match_in_magnitude():
    err, strips = setup()
    got = {}
    for q in (2, 4, 8):
        got[q] = err(orc.coarse_sequential(strips(q, 1 / 32), T, N, 1, s, np.zeros((n, n))))
    pr = GOLD["printed"]["coarse_error"]
    assert abs(got[2] / pr["2"] - 1) < 0.05 and abs(got[4] / pr["4"] - 1) < 0.02, got
    assert 0.5 < got[8] / pr["8"] < 2.0, got


@pytest.mark.slow
def test_parareal_five_iterations_q2_magnitude():
    err, strips = setup()
    U, _, it = orc.parareal(strips(2, 1 / 16), T, N, 1, s, np.zeros((n, n)), 0.0, max_iter=5,
                            pG=strips(2, 1 / 32))
    assert it == 5
    e = err(U)
    pr = GOLD["printed"]["parareal_error_after_5_iterations"]["2"]
    assert 0.5 < e / pr < 2.0, e
    # the five-iteration error is of the fine error's order, the paper's point
    assert e < 2 * GOLD["printed"]["fine_error"]
