"""Writes the stored expected values of tests/golden/ with the CPU oracle only.

c1_laplace2d_n1024.json -- the n = 1024 unit-square Laplace workload
(A_ij = 1/(|x_i - x_j| + 1e-3), Sec. 5.1's kernel, points from
workloads.uniform_cube(1024, 2, seed 1)): dense eigenvalues lambda_500..524
(LAPACK, Sec. 5's dsyev comparison), Gershgorin interval, ||A||_inf, and the
H^2 oracle's lambda~_512 by Algorithm 1 at eps_ev = 1e-8 (leaf 64, rank 16,
eta 1, eps_H2 = 1e-10) with ||A - A~||_2.

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import dense, h2  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def c1():
    n, seed = 1024, 1
    X = W.uniform_cube(n, 2, seed)
    kp = (1e-3, 0.0, 0.0, 0.0)
    A = dense.kernel_matrix(W.LAPLACE_EPS, kp, X)
    ev = dense.eigenvalues(A)
    ga, gb = dense.gershgorin(A)
    h = h2.construct(X, W.LAPLACE_EPS, kp, 64, 16, 1.0, eps_h2=1e-10)
    At = h2.dense_approximation(h)
    err = float(np.linalg.norm(dense.kernel_matrix(W.LAPLACE_EPS, kp, h.X) - At, 2))
    mids, lo, hi, evals = h2.kth_eigenvalues(h, [512], 1e-8)
    return {
        "workload": "laplace2d n=1024 seed=1 leaf=64 rank=16 eta=1 eps_h2=1e-10",
        "citation": "Sec. 5.1 (kernel 1/(|x_i-x_j|+1e-3)); Algorithm 1; Eq. error-bound",
        "dense_eigs_500_524": [float(v) for v in ev[499:524]],
        "gershgorin": [ga, gb],
        "norm_inf": float(np.max(np.sum(np.abs(A), axis=1))),
        "norm2": float(np.max(np.abs(ev))),
        "h2_err2": err,
        "h2_lambda_512_tol1e-8": mids[0],
        "h2_interval_512": [lo[0], hi[0]],
        "h2_evals": evals,
        "max_rank": h.stats["max_rank"],
    }


if __name__ == "__main__":
    out = c1()
    with open(os.path.join(HERE, "c1_laplace2d_n1024.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))
