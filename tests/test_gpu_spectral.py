"""The Fourier spectral BdG operator and solves on the GPU (Section 4,
Example "large-scale dense matrix", eq. bdg_KM, Table 8), through the C ABI.

* products: the per-axis FFT kernels against the oracle's 3-D FFT, on grids
  with flat axes, every line length 2..256, ragged column counts and a
  leading dimension > n; float64 within a few units of the FFT's normwise
  rounding bound, float32 transforms (mixed-precision CG products) within
  the float32 one;
* solves: 16^3 against the oracle's definition route (1e-10 relative);
  32^3 and 64^3 against Table 8 and the analytic eigenpairs gamma_alpha;
  mixed precision against the float64 solve; nullspace discovery finds phi_s.
"""
import math

import numpy as np
import pytest

from conftest import from_dev, load_golden, to_dev
from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def L(built_lib):
    from paper_2506_08355_gb300 import lrep
    return lrep


def _scale(dims, lengths, coef, d, X):
    """max |multiplier| summed over the axes plus max |d|, times max |X|."""
    mu = sum(abs(coef) * (math.pi * N / Ld) ** 2 for N, Ld in zip(dims, lengths) if N > 1)
    return (mu + np.abs(d).max()) * np.abs(X).max()


@pytest.mark.parametrize("dims,c", [((16, 16, 16), 16), ((32, 8, 4), 3), ((64, 1, 1), 17),
                                    ((1, 32, 1), 5), ((1, 1, 16), 2), ((2, 2, 2), 1),
                                    ((256, 4, 2), 7), ((8, 16, 32), 9), ((4, 128, 2), 4),
                                    ((1, 1, 1), 3)])
def test_spectral_apply_parity(L, dims, c):
    import torch
    rng = np.random.default_rng(sum(dims) + c)
    lengths = (16.0, 11.0, 7.0)
    n = int(np.prod(dims))
    dK, dM = rng.standard_normal(n), rng.uniform(1.0, 2.0, n)
    op = R.SpectralOp(*dims, lengths, -0.5, dK, dM)
    X = rng.standard_normal((n, c))
    prob = L.Problem.spectral(*dims, lengths, -0.5, dK, dM)
    ld = n + 5
    Xd = torch.zeros((c, ld), dtype=torch.float64, device="cuda")
    Xd[:, :n] = torch.from_numpy(X.T.copy()).cuda()
    Yd = torch.full((c, ld), 7.0, dtype=torch.float64, device="cuda")
    Xv, Yv = Xd[:, :n], Yd[:, :n]
    logn = max([int(math.log2(N)) for N in dims] + [1])
    for op_id, w, d in ((L.OP_K, "K", dK), (L.OP_M, "M", dM)):
        ref = op.apply(w, X)
        prob.apply(op_id, Xv, Yv)
        got = Yd[:, :n].cpu().numpy().T
        assert np.abs(got - ref).max() <= 8 * logn * U * _scale(dims, lengths, -0.5, d, X)
        # the padding past n is left alone
        assert torch.all(Yd[:, n:] == 7.0)
    prob.close()


def test_spectral_apply_float32_transforms(L):
    """The CG products of the mixed precision mode: float32 transforms."""
    import torch
    dims, lengths = (32, 32, 32), (16.0, 16.0, 16.0)
    p = synth.bdg_spectral(32)
    op = R.SpectralOp(*dims, lengths, -0.5, p["dK"], p["dM"])
    X = np.random.default_rng(5).standard_normal((p["n"], 16))
    prob = L.Problem.spectral(*dims, lengths, -0.5, p["dK"], p["dM"])
    prob.set_options(precision=L.PREC_MIXED_BF16X3)
    Y = L.device_block(p["n"], 16)
    Y64 = L.device_block(p["n"], 16)
    for op_id, w, d in ((L.OP_K, "K", p["dK"]), (L.OP_M, "M", p["dM"])):
        ref = op.apply(w, X)
        prob.apply(op_id, to_dev(X), Y, cg=True)
        prob.apply(op_id, to_dev(X), Y64)
        err32 = np.abs(from_dev(Y) - ref).max()
        err64 = np.abs(from_dev(Y64) - ref).max()
        sc = _scale(dims, lengths, -0.5, d, X)
        assert err32 <= 8 * 5 * 2.0 ** -24 * sc
        assert err64 <= 8 * 5 * U * sc
        assert err32 > 10 * err64  # the CG product really ran in float32
    prob.close()


def _problem(L, N, prec=None):
    p = synth.bdg_spectral(N)
    prob = L.Problem.spectral(N, N, N, p["lengths"], p["lap_coef"], p["dK"], p["dM"])
    prob.set_nullspace(p["phi"][:, None])
    if prec is not None:
        prob.set_options(precision=prec)
    return p, prob


def _check_pairs(L, p, prob, tol, nev):
    assert prob.nconv() == nev
    lam = prob.eigvals()
    op = R.SpectralOp(p["nx"], p["ny"], p["nz"], p["lengths"], p["lap_coef"], p["dK"],
                      p["dM"])
    X, Y = prob.vectors(), prob.vectors(which=L.Q_Y)
    res = R.residuals(op, X, Y, lam)
    assert res.max() < tol, res.max()
    np.testing.assert_allclose(X.T @ Y, np.eye(nev), atol=1e-12)
    # deflation: phi_s^T K x = lam phi_s^T y = 0, so every y is orthogonal to
    # the null vector phi_s
    assert np.abs(p["phi"] @ Y).max() < 1e-10
    return lam, X, Y


def test_bdg16_fp64_vs_definition(L):
    """n = 16^3: FP64 solve against the oracle's definition route."""
    p, prob = _problem(L, 16)
    assert prob.solve(8, 8, 1e-10) == L.OK
    lam, X, Y = _check_pairs(L, p, prob, 1e-10, 8)
    op = R.SpectralOp(16, 16, 16, p["lengths"], -0.5, p["dK"], p["dM"])
    K = op.apply("K", np.eye(4096))
    M = op.apply("M", np.eye(4096))
    K, M = 0.5 * (K + K.T), 0.5 * (M + M.T)
    kap, Vk = np.linalg.eigh(K)
    FK = Vk[:, 1:] * np.sqrt(kap[1:])[None, :]
    ref = R.lrep_definition_values(FK, np.linalg.cholesky(M), 8)
    np.testing.assert_allclose(lam, ref, rtol=1e-10)
    prob.close()


@pytest.mark.parametrize("N,col", [(32, 2), (64, 3)])
def test_bdg_table8(L, N, col):
    """32^3 and 64^3 (h0/2, h0/4): Table 8's values, tol 1e-8 as in the paper."""
    tab = load_golden("table8_bdg.txt")[:, col]
    p, prob = _problem(L, N)
    assert prob.solve(8, 8, 1e-8) == L.OK
    lam, X, Y = _check_pairs(L, p, prob, 1e-8, 8)
    np.testing.assert_allclose(lam, tab, rtol=0, atol=1e-9)
    if N == 64:
        # analytic eigenpairs gamma_alpha (x: K-side alpha phi_s, y: M-side
        # d_alpha phi_s): lambda_1 = lambda_2 = 1, lambda_6 = 2 to 1e-8, and
        # pair 6 is the z mode: X_6 parallel to z phi_s
        assert abs(lam[0] - 1.0) < 1e-8 and abs(lam[1] - 1.0) < 1e-8
        assert abs(lam[5] - 2.0) < 1e-8
        z = (-8.0 + np.arange(N) * 16.0 / N)[:, None, None] * np.ones((N, N, N))
        g = (z.reshape(-1) * p["phi_s"])
        cos = abs(g @ X[:, 5]) / (np.linalg.norm(g) * np.linalg.norm(X[:, 5]))
        assert 1.0 - cos < 1e-6, 1.0 - cos
    prob.close()


@pytest.mark.parametrize("prec_name", ["PREC_MIXED_BF16X3", "PREC_MIXED_SLICED"])
def test_bdg32_mixed_matches_fp64(L, prec_name):
    """Mixed precision (float32 transforms in the CG products): the same
    eigenvalues as the FP64 solve, every residual below tol."""
    p, prob = _problem(L, 32)
    assert prob.solve(8, 8, 1e-8) == L.OK
    lam64 = prob.eigvals()
    prob.set_options(precision=getattr(L, prec_name))
    assert prob.solve(8, 8, 1e-8) == L.OK
    lam, X, Y = _check_pairs(L, p, prob, 1e-8, 8)
    np.testing.assert_allclose(lam, lam64, rtol=1e-10)
    prob.close()


def test_bdg16_find_nullspace(L):
    """Nullspace discovery on the spectral operator: N(K) = span(phi_s), then
    the solve at the paper's tol 1e-8 (the discovered basis is exact to its
    residual tolerance, which bounds the residuals a solve can reach)."""
    p = synth.bdg_spectral(16)
    prob = L.Problem.spectral(16, 16, 16, p["lengths"], -0.5, p["dK"], p["dM"])
    X0, its = prob.find_nullspace(r_max=4, tol=1e-12)
    assert X0.shape == (4096, 1)
    assert abs(abs(p["phi"] @ X0[:, 0]) - 1.0) < 1e-12
    assert prob.solve(8, 8, 1e-8) == L.OK
    tab = load_golden("table8_bdg.txt")[:, 1]
    np.testing.assert_allclose(prob.eigvals(), tab, rtol=0, atol=2e-10)
    prob.close()


def test_spectral_rejects_bad_grid(L):
    with pytest.raises(L.LrepError):
        L.Problem.spectral(24, 16, 16, (16.0, 16.0, 16.0), -0.5, np.zeros(24 * 256),
                           np.ones(24 * 256))
    with pytest.raises(L.LrepError):
        L.Problem.spectral(512, 1, 1, (16.0, 16.0, 16.0), -0.5, np.zeros(512), np.ones(512))
