"""Writes fig10_oracle_errors.json: the oracle's errors for the Sec. 5.2 experiment of Fig. 10 at
h = 1/64 (63^2 interior nodes), T = 1, Delta T = 0.05 (N = 20), two subdomains of one strip
each with overlap 1/16, the manufactured full-tensor problem: max over the coarse times of the
h-weighted 2-norm of the difference between the parareal iterate after k iterations and the
fine solution, for Parareal/FIE-FIE (k = 4) and Parareal/FIE-DR (k = 5, 6) with s = 2, 4, 10.

Calls only the oracle and the seeded input recipes (no GPU code).  Run from the repository
root:  python tests/golden/make_fig10_oracle.py   (about two minutes on the host cores).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
from paper_2502_08370_gb300 import workloads as wl  # noqa: E402

n, T, N = 63, 1.0, 20


def errors(fine, s, ks):
    h = 1.0 / (n + 1)
    m = wl.manufactured_full_tensor((n, n), T, N, s)
    p = orc.Problem((n, n), a=m["a"], d12=m["d12"], split="dd", boxes=(2, 1), overlap=1 / 16, src=m["src"],
                    src_t=m["src_t"], src2=m["src2"], src2_t=m["src2_t"])
    u0 = np.zeros((n, n))
    F = orc.fine_sequential_dr(p, T, N, s, u0) if fine == "dr" else orc.fine_sequential(p, T, N, s, u0)
    out = {}
    for k in ks:
        U, _, it = orc.parareal(p, T, N, 1, s, u0, 0.0, max_iter=k, fine=fine)
        assert it == k
        out[str(k)] = max(float(np.sqrt(h * h * np.sum((U[j] - F[j]) ** 2))) for j in range(1, N + 1))
    return out


def main():
    res = {"source": "oracle/ (FP64), written by tests/golden/make_fig10_oracle.py",
           "setup": {"n": n, "T": T, "N": N, "boxes": [2, 1], "overlap": 1 / 16, "problem": "manufactured_full_tensor"},
           "fie": {str(s): errors("fie", s, [4]) for s in (2, 4, 10)},
           "dr": {str(s): errors("dr", s, [5, 6]) for s in (2, 4, 10)}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fig10_oracle_errors.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=2)
        f.write("\n")
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
