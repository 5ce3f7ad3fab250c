"""Writes the stored expected values of the full-size workloads.

Calls only the oracle and the seeded input generators:
    python tests/golden/make_golden.py config1
config1: the 64 smallest positive eigenvalues of the dense n = 8192
workload with a 4-dimensional nullspace of K (definition route, values
only, with the construction's factors F_K = Q1 diag(sqrt k),
F_M = Q2 diag(sqrt m)).
config3: the 256 smallest positive eigenvalues of the dense n = 32768
mixed-precision workload (k, m log-uniform in [1e-2, 1e2], Haar Q1, Q2 in
Householder form, seed 3), by the same values-only definition route from
the factors F_K = Q1 diag(sqrt k), F_M = Q2 diag(sqrt m).  About 1.5 h on
8 cores and ~40 GB of host memory (two dorgqr, one GEMM and one
values-only SVD of order 32768).
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


def config3():
    import time
    t0 = time.perf_counter()
    g = synth.loguniform_reflected(32768, seed=3)
    FK = synth.reflected_factor_host(g["V1"], g["tau1"], g["sgn1"], g["k"])
    del g["V1"]
    FM = synth.reflected_factor_host(g["V2"], g["tau2"], g["sgn2"], g["m"])
    del g["V2"]
    t1 = time.perf_counter()
    lam = R.lrep_definition_values(FK, FM, 256)
    dt = time.perf_counter() - t0
    path = os.path.join(HERE, "config3_lambda.txt")
    with open(path, "w") as f:
        f.write("# 256 smallest positive eigenvalues of the dense n = 32768 workload\n"
                "# (synth.loguniform_reflected(32768, seed=3): Haar Q1, Q2 in Householder\n"
                "# form, k, m log-uniform in [1e-2, 1e2]), definition route of the oracle\n"
                "# (values-only SVD of F_K^T F_M); factors %.0f s, total %.0f s; written by\n"
                "# tests/golden/make_golden.py config3\n" % (t1 - t0, dt))
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
