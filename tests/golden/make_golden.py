"""Writes the stored expected values of the full-size workloads.

Calls only the oracle and the seeded input generators:
    python tests/golden/make_golden.py config1
config1: the 64 smallest positive eigenvalues of the dense n = 8192
workload with a 4-dimensional nullspace of K (definition route, values
only, with the construction's factors F_K = Q1 diag(sqrt k),
F_M = Q2 diag(sqrt m)).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lrep_ref as R  # noqa: E402
from paper_2506_08355_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def config1():
    p = synth.config(1)
    FK = p["Q1"] * np.sqrt(p["k"])[None, :]
    FM = p["Q2"] * np.sqrt(p["m"])[None, :]
    lam = R.lrep_definition_values(FK, FM, p["nev"], r=p["r"])
    path = os.path.join(HERE, "config1_lambda.txt")
    with open(path, "w") as f:
        f.write("# 64 smallest positive eigenvalues of the dense n = 8192 workload\n"
                "# (synth.config(1): Haar Q1, Q2 seed 1, k, m ~ U[0.5, 10], 4 zero k),\n"
                "# definition route of the oracle (values-only SVD); written by\n"
                "# tests/golden/make_golden.py config1\n")
        for v in lam:
            f.write("%.17e\n" % v)
    print(path)


def config1_r2():
    """Full literal Alg. 2 (oracle R2) on the same workload: iteration and
    product counts, and the eigenvalues it returns."""
    import time
    p = synth.config(1)
    op = R.DenseOp(p["K"], p["M"])
    t0 = time.perf_counter()
    res = R.bosp(op, p["nev"], p["block"], p["tol"], X0=p["X0"])
    dt = time.perf_counter() - t0
    path = os.path.join(HERE, "config1_oracle_run.txt")
    with open(path, "w") as f:
        f.write("# oracle R2 (literal Alg. 2, numpy FP64) on synth.config(1):\n"
                "# n = 8192, nev = 64, nb = 16, tol 1e-10, 4-dim nullspace; written by\n"
                "# tests/golden/make_golden.py config1_r2\n")
        f.write("iters %d\nmatvecs %d\nconverged %d\nrebiorths %d\nseconds %.1f\n"
                % (res.iters, res.matvecs, int(res.converged), res.rebiorths, dt))
        for v in res.lam:
            f.write("lam %.17e\n" % v)
    print(path)


def config2_r2():
    """Oracle R2 (literal Alg. 2) on the 64^3 BdG-like stencil workload:
    n = 262144, nev = 32, nb = 16, tol 1e-10, nullspace phi."""
    import time
    p = synth.config(2)
    op = R.StencilOp(p["nx"], p["ny"], p["nz"], p["h"], -0.5, p["dK"], p["dM"])
    t0 = time.perf_counter()
    res = R.bosp(op, p["nev"], p["block"], p["tol"], X0=p["X0"])
    dt = time.perf_counter() - t0
    path = os.path.join(HERE, "config2_oracle_run.txt")
    with open(path, "w") as f:
        f.write("# oracle R2 (literal Alg. 2, numpy FP64) on synth.config(2):\n"
                "# 64^3 BdG-like 7-point stencil, nev = 32, nb = 16, tol 1e-10,\n"
                "# nullspace phi; written by tests/golden/make_golden.py config2_r2\n")
        f.write("iters %d\nmatvecs %d\nconverged %d\nrebiorths %d\nseconds %.1f\n"
                % (res.iters, res.matvecs, int(res.converged), res.rebiorths, dt))
        for v in res.lam:
            f.write("lam %.17e\n" % v)
    print(path)


if __name__ == "__main__":
    for name in sys.argv[1:] or ["config1"]:
        globals()[name]()
