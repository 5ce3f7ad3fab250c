"""Generalized LREP (Remark on the generalized LREP): K x = lam B y,
M y = lam B x with an SPD mass matrix B, solved by Alg. 2 in the
B-inner product on the GPU.  Compared with the definition route through
B = L L^T (oracle), residuals re-checked on the CPU with B, and X^T B Y = I.
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


def _problem(n, r, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q3, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = rng.uniform(0.5, 10, n)
    k[:r] = 0.0
    K = (Q1 * k) @ Q1.T
    M = (Q2 * rng.uniform(0.5, 10, n)) @ Q2.T
    Bm = (Q3 * rng.uniform(0.5, 2.0, n)) @ Q3.T
    return K, M, Bm, Q1[:, :r].copy()


def _check(L, prob, K, M, Bm, nev, r, tol, rtol=1e-10, vectors=True):
    lam_d, Xd, Yd = R.lrep_definition_gen(K, M, Bm, nev, r)
    assert prob.nconv() == nev
    lam = prob.eigvals()
    np.testing.assert_allclose(lam, lam_d, rtol=rtol)
    X, Y = prob.vectors(), prob.vectors(which=L.Q_Y)
    op = R.DenseOp(K, M, Bm)
    res = R.residuals(op, X, Y, lam)
    assert res.max() < tol, res.max()
    np.testing.assert_allclose(prob.residuals(), res, rtol=1e-6, atol=1e-14)
    np.testing.assert_allclose(X.T @ Bm @ Y, np.eye(nev), atol=1e-11)
    if vectors:  # unique up to sign for a simple spectrum
        np.testing.assert_allclose(np.abs(X), np.abs(Xd), atol=1e-7)
    return lam, X, Y


@pytest.mark.parametrize("n,nev,nb,r,prec", [(200, 4, 4, 0, 0), (600, 12, 4, 0, 0),
                                             (500, 8, 4, 2, 0), (700, 8, 4, 2, 3)])
def test_generalized_dense(L, n, nev, nb, r, prec):
    K, M, Bm, X0 = _problem(n, r, 50 + n + r)
    prob = L.Problem.dense(K, M)
    prob.set_mass(Bm)
    prob.set_options(precision=prec)
    if r:
        prob.set_nullspace(X0)
    assert prob.solve(nev, nb, 1e-10) == L.OK
    lam, X, Y = _check(L, prob, K, M, Bm, nev, r, 1e-10)
    if r:
        assert np.abs(X0.T @ Bm @ Y).max() < 1e-9
    prob.close()


def test_generalized_csr_mass(L):
    """CSR K, M (the BdG-like stencil on a 10^3 grid) with a lumped-plus-
    coupling mass matrix B given in CSR form."""
    s = synth.bdg_stencil(10)
    n = s["n"]
    rpK, ciK, vK = synth.stencil_to_csr(s["nx"], s["ny"], s["nz"], s["h"], -0.5, s["dK"])
    rpM, ciM, vM = synth.stencil_to_csr(s["nx"], s["ny"], s["nz"], s["h"], -0.5, s["dM"])
    # B = I + 0.1 * (normalised graph Laplacian of the grid): SPD, CSR
    rpL, ciL, vL = synth.stencil_to_csr(s["nx"], s["ny"], s["nz"], 1.0, 1.0, np.zeros(n))
    vB = -0.1 * vL / 6.0
    rows = np.repeat(np.arange(n), np.diff(rpL))
    vB[ciL == rows] += 1.0
    def todense(rp, ci, v):
        A = np.zeros((n, n))
        np.add.at(A, (np.repeat(np.arange(n), np.diff(rp)), ci), v)
        return A
    K, M, Bm = todense(rpK, ciK, vK), todense(rpM, ciM, vM), todense(rpL, ciL, vB)
    X0 = s["phi"][:, None] / np.linalg.norm(s["phi"])
    prob = L.Problem.csr(n, (rpK, ciK, vK), (rpM, ciM, vM))
    prob.set_mass((rpL, ciL, vB))
    prob.set_nullspace(X0)
    assert prob.solve(8, 4, 1e-10) == L.OK
    # the trap is symmetric in x and y: degenerate pairs, vectors not unique
    _check(L, prob, K, M, Bm, 8, 1, 1e-10, vectors=False)
    prob.close()
