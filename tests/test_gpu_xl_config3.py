"""The mixed-precision workload at full size: dense n = 32768, K = Q1 diag(k)
Q1^T, M = Q2 diag(m) Q2^T with Haar Q1, Q2 (Householder form, seed 3) and
k, m log-uniform in [1e-2, 1e2]; nev = 256 in moving-window batches of 32,
tol 1e-8.  The wanted pairs are a cluster at the bottom of a spectrum four
decades wide, so the CG budget of eq. block_GS is 100 iterations.

Expected values: the 256 smallest positive eigenvalues of the oracle's
definition route (values-only SVD of F_K^T F_M from the construction's
factors), stored by tests/golden/make_golden.py config3.  The device forms
K = F_K F_K^T, M = F_M F_M^T from the same Householder draws; forming them
perturbs the eigenvalues by ~1e-13 relative (tests/test_synth_haar.py ties
the two routes at small n).

Bar, in the mixed-precision mode (bf16 hi/lo CG products, every product
entering H^ float64-accurate) and in the FP64 mode (every product
float64-accurate by error-free slicing): every eigenvalue within 1e-10
relative of the stored values, every residual of eq. tol recomputed on the
CPU in float64 below tol, X^T Y = I to 1e-12.  The per-eigenpair error of
both modes is printed (pytest -s).
"""
import numpy as np
import pytest

from conftest import load_golden
from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth

pytestmark = pytest.mark.gpu

N, NEV, NB, TOL, CG = 32768, 256, 32, 1e-8, 100


@pytest.fixture(scope="module")
def L(built_lib):
    from paper_2506_08355_gb300 import lrep
    return lrep


@pytest.fixture(scope="module")
def workload():
    import torch
    g = synth.loguniform_reflected(N, seed=3)
    K = synth.reflected_operator_device(g["V1"], g["tau1"], g["sgn1"], g["k"])
    M = synth.reflected_operator_device(g["V2"], g["tau2"], g["sgn2"], g["m"])
    del g
    torch.cuda.synchronize()
    op = R.DenseOp(K.cpu().numpy(), M.cpu().numpy())
    yield K, M, op, load_golden("config3_lambda.txt")
    del K, M
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec_name", ["PREC_MIXED_SLICED", "PREC_FP64_SLICED"])
def test_config3_full_size(L, workload, prec_name):
    K, M, op, lam_ref = workload
    prob = L.Problem.dense(K, M, borrow=True)
    prob.set_options(precision=getattr(L, prec_name), cg_maxit=CG, maxit=3000)
    assert prob.solve(NEV, NB, TOL) == L.OK
    assert prob.nconv() == NEV
    lam = prob.eigvals()
    rel = np.abs(lam - lam_ref) / lam_ref
    X, Y = prob.vectors(), prob.vectors(which=L.Q_Y)
    res = R.residuals(op, X, Y, lam)
    E = np.abs(X.T @ Y - np.eye(NEV))
    bio = E.max()
    # within each batch of 64 locked pairs and across batches
    blk = np.kron(np.eye(NEV // 64), np.ones((64, 64))) > 0
    print("\n%s: max |X^T Y - I| within batches %.2e, across batches %.2e"
          % (prec_name, E[blk].max(), E[~blk].max()))
    print("\n%s: %d outer iterations; eigenvalue error vs definition route: max %.2e, "
          "median %.2e; max residual %.2e; max |X^T Y - I| %.2e"
          % (prec_name, prob.iters(), rel.max(), np.median(rel), res.max(), bio))
    print("%s per-eigenpair relative error: %s" % (
        prec_name, " ".join("%.1e" % v for v in rel)))
    assert rel.max() < 1e-10, rel.max()
    assert res.max() < TOL, res.max()
    np.testing.assert_allclose(prob.residuals(), res, rtol=1e-6, atol=1e-14)
    assert bio < 1e-12
    prob.close()
