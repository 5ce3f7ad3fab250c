"""Nullspace discovery on the GPU (lrep_find_nullspace): the pre-step of the
Remark on the numerical computation of the generalized nullspace.

The basis is not unique; its orthogonal projector is.  Each case compares
the projector with the oracle's (the definition: eigenvectors of K for
eigenvalues <= tol ||K||), checks the dimension and ||K X0||.
"""
import numpy as np
import pytest

from conftest import load_golden
from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth
from test_gpu_solver import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(built_lib):
    from paper_2506_08355_gb300 import lrep
    return lrep


def _dense_with_kernel(n, r, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = rng.uniform(0.5, 10.0, n)
    k[:r] = 0.0
    m = rng.uniform(0.5, 10.0, n)
    return (Q * k) @ Q.T, (Q * m) @ Q.T


@pytest.mark.parametrize("n,r", [(1000, 4), (777, 1), (600, 0)])
def test_find_nullspace_dense(L, n, r):
    K, M = _dense_with_kernel(n, r, 40 + r)
    prob = L.Problem.dense(K, M)
    X0, its = prob.find_nullspace(r_max=8, tol=1e-10)
    ref, w = R.nullspace_definition(K, 1e-10)
    assert ref.shape[1] == r and X0.shape == (n, r)
    np.testing.assert_allclose(X0 @ X0.T, ref @ ref.T, atol=1e-8)
    np.testing.assert_allclose(X0.T @ X0, np.eye(r), atol=1e-12)
    if r:
        assert np.abs(K @ X0).max() <= 1e-9 * np.abs(w).max()
    prob.close()


def test_find_nullspace_stencil(L):
    """16^3 BdG-like stencil: K's kernel is the Gaussian phi (1-dim)."""
    s = synth.bdg_stencil(16)
    prob = L.Problem.stencil(s["nx"], s["ny"], s["nz"], s["h"], -0.5, s["dK"], s["dM"])
    X0, its = prob.find_nullspace(r_max=4, tol=1e-10)
    assert X0.shape == (s["n"], 1)
    phi = s["phi"] / np.linalg.norm(s["phi"])
    assert abs(abs(phi @ X0[:, 0]) - 1.0) < 1e-9
    prob.close()


def test_find_nullspace_rejects_too_small_rmax(L):
    K, M = _dense_with_kernel(300, 6, 5)
    prob = L.Problem.dense(K, M)
    with pytest.raises(L.LrepError):
        prob.find_nullspace(r_max=1, tol=1e-10)
    prob.close()


def test_discovered_nullspace_full_size_solve(L):
    """n = 8192 workload without a caller-supplied X0: discovery, then the
    solve; same eigenvalues as the stored definition-route values."""
    g = load_golden("config1_lambda.txt")
    p = synth.config(1)
    prob = L.Problem.dense(p["K"], p["M"])
    X0, its = prob.find_nullspace(r_max=8, tol=1e-10)
    assert X0.shape[1] == 4
    Pt = p["X0"] @ np.linalg.pinv(p["X0"])
    np.testing.assert_allclose(X0 @ X0.T, Pt, atol=1e-8)
    assert prob.solve(64, 16, 1e-10) == L.OK
    check(R.DenseOp(p["K"], p["M"]), prob, g, 1e-10, 64)
    prob.close()
