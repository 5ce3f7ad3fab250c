"""The mixed-precision workload with log-uniform spectra (k, m in [1e-2, 1e2],
Haar Q1, Q2) at a size the oracle's definition route finishes in seconds:
n = 2048, nev = 32 in moving windows of 16, tol 1e-8.  The wanted pairs sit
in a cluster at the bottom of a spectrum three decades wide (relative gaps
~1e-3), the hard case for the inexact CG products.

Bar: every precision converges; eigenvalues within 1e-9 relative of the
definition route (the float64 mode and the mixed modes alike), residuals
recomputed on the CPU below tol, X^T Y = I to 1e-12.
"""
import numpy as np
import pytest

from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(built_lib):
    from paper_2506_08355_gb300 import lrep
    return lrep


@pytest.fixture(scope="module")
def problem():
    p = synth.haar_dense(2048, seed=3, k_range=(1e-2, 1e2), m_range=(1e-2, 1e2),
                         law="loguniform")
    lam, _, _ = R.lrep_definition(p["K"], p["M"], 32)
    return p, lam


@pytest.mark.parametrize("prec_name", ["PREC_FP64", "PREC_MIXED_BF16X3", "PREC_MIXED_SLICED",
                                       "PREC_FP64_SLICED"])
def test_loguniform_n2048(L, problem, prec_name):
    p, lam_ref = problem
    prob = L.Problem.dense(p["K"], p["M"])
    prob.set_options(precision=getattr(L, prec_name), maxit=3000)
    assert prob.solve(32, 16, 1e-8) == L.OK
    lam = prob.eigvals()
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-9)
    X, Y = prob.vectors(), prob.vectors(which=L.Q_Y)
    res = R.residuals(R.DenseOp(p["K"], p["M"]), X, Y, lam)
    assert res.max() < 1e-8, res.max()
    np.testing.assert_allclose(X.T @ Y, np.eye(32), atol=1e-12)
    print("%s: %d outer iterations, max rel eig err %.2e, max residual %.2e"
          % (prec_name, prob.iters(), np.max(np.abs(lam - lam_ref) / lam_ref), res.max()))
    prob.close()
