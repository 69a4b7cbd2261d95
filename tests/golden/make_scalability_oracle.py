"""Writes scalability_oracle_errors.json: the oracle's errors for the scalability experiment of
Sec. 5.1 (h = 0.01, T = 1, DeltaT = 1/32, delta t = 1/3200; fine DD with q = 2 strips of
overlap 1/16, coarse DD with q = 2, 4, 8 strips of overlap 1/32; five parareal iterations
from u = 0), measured like the paper: max over the coarse times of the h-weighted 2-norm of the
error against the manufactured solution u = sin(2 pi t) sin(2 pi x) sin(2 pi y).

Calls only the oracle and the seeded input recipes (no GPU code).  Run from the repository
root:  python tests/golden/make_scalability_oracle.py   (a few minutes on the host cores).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_2502_08370_gb300 import workloads as wl  # noqa: E402

n, T, N, s = 99, 1.0, 32, 100


def main():
    S, st, exact = wl.manufactured((n, n), T, N, s)
    h = 1.0 / (n + 1)

    def err(U):
        return max(float(np.sqrt(h * h * np.sum((U[j] - exact(j * T / N)) ** 2))) for j in range(1, N + 1))

    def strips(q, beta):
        return orc.Problem((n, n), src=S, src_t=st, split="dd", boxes=(2 * q, 1), overlap=beta)

    u0 = np.zeros((n, n))
    out = {"source": "oracle/ (FP64), written by tests/golden/make_scalability_oracle.py",
           "setup": {"n": n, "T": T, "N": N, "s": s, "fine": {"q": 2, "beta": 1 / 16},
                     "coarse_beta": 1 / 32, "iterations": 5},
           "fine_error": err(orc.fine_sequential(strips(2, 1 / 16), T, N, s, u0)),
           "coarse_error": {}, "parareal_error_after_5_iterations": {}}
    for q in (2, 4, 8):
        out["coarse_error"][str(q)] = err(orc.coarse_sequential(strips(q, 1 / 32), T, N, 1, s, u0))
        U, _, it = orc.parareal(strips(2, 1 / 16), T, N, 1, s, u0, 0.0, max_iter=5, pG=strips(q, 1 / 32))
        assert it == 5
        out["parareal_error_after_5_iterations"][str(q)] = err(U)
        print(q, out["coarse_error"][str(q)], out["parareal_error_after_5_iterations"][str(q)], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scalability_oracle_errors.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
