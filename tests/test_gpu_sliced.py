"""Float64-accurate dense products by error-free slicing on the bf16 tensor
cores (precision FP64_SLICED / MIXED_SLICED).

The product's bound has the form of the float64 product's own:
|Y_ij - (A X)_ij| <= c n u 2^(e_i + f_j) with 2^e_i > max_k |A_ik| and
2^f_j > max_k |X_kj|.  In the worst case (every digit truncation of the
same sign) c ~ 2^-1.7; on random inputs the errors cancel like those of a
float64 dot product and c ~ 1e-3.  The tests check c <= 1/8 against the
EXACT dot product (rational arithmetic on the float64 inputs), a bound that
a dropped or mis-weighted level, a wrong scale or a transposed operand all
exceed by orders of magnitude.  Inputs whose float64 product is exact must
come out bit-exact.
"""
import math

import numpy as np
import pytest

from conftest import load_golden
from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth
from test_gpu_solver import check

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def L(built_lib):
    from paper_2506_08355_gb300 import lrep
    return lrep


def _apply(L, A, X, prec=2):
    import torch
    n = A.shape[0]
    prob = L.Problem.dense(A, A)
    prob.set_options(precision=prec)
    Xd = torch.tensor(np.ascontiguousarray(X.T), device="cuda")
    Yd = torch.full_like(Xd, np.nan)
    prob.apply(L.OP_K, Xd, Yd)
    torch.cuda.synchronize()
    prob.close()
    return Yd.cpu().numpy().T


def _exact_dot(a, x):
    """sum_k a_k x_k exactly, as (numerator, 2-power denominator)."""
    terms = []
    for ai, xi in zip(a.tolist(), x.tolist()):
        p, q = ai.as_integer_ratio()
        r, s = xi.as_integer_ratio()
        terms.append((p * r, q * s))
    den = max(d for _, d in terms)
    return sum(nu * (den // d) for nu, d in terms), den


def _err(y, exact):
    num, den = exact
    p, q = float(y).as_integer_ratio()
    return abs(p * den - num * q) / (q * den)


@pytest.mark.parametrize("c", [1, 5, 16, 17, 40])
def test_sliced_product_exact_on_short_mantissas(L, c):
    """Entries with few significant bits: float64 A X is exact, and so must
    the sliced product be (2 digits per value, every level sum exact)."""
    rng = np.random.default_rng(100 + c)
    n = 1000  # 7 full row tiles + 104, 15 full k-tiles + 40
    A = rng.integers(-1024, 1025, (n, n)).astype(np.float64) * 2.0 ** -10
    A = np.triu(A) + np.triu(A, 1).T
    X = rng.integers(-4096, 4097, (n, c)).astype(np.float64) * 2.0 ** -3
    Y = _apply(L, A, X)
    np.testing.assert_array_equal(Y, A @ X)


@pytest.mark.parametrize("law,c", [("normal", 16), ("wide", 16), ("normal", 32), ("wide", 7)])
def test_sliced_product_error_bound(L, law, c):
    rng = np.random.default_rng(7 + c + (law == "wide"))
    n = 1500
    if law == "normal":
        A = rng.standard_normal((n, n))
        X = rng.standard_normal((n, c))
    else:  # entries spread over ~35 binades, rows and columns of unequal scale
        A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-12, 12, (n, n)))
        X = rng.standard_normal((n, c)) * np.exp(rng.uniform(-6, 6, (n, c)))
    A = (A + A.T) / 2
    Y = _apply(L, A, X)
    assert np.all(np.isfinite(Y))
    worst = 0.0
    for i in rng.choice(n, 24, replace=False):
        e = math.frexp(np.abs(A[i]).max())[1]
        for j in range(c):
            f = math.frexp(np.abs(X[:, j]).max())[1]
            scale = n * U * 2.0 ** (e + f)
            worst = max(worst, _err(Y[i, j], _exact_dot(A[i], X[:, j])) / scale)
    assert worst <= 1.0 / 8, worst
    # and the whole block against float64 (whose own error has the same form)
    ref = A @ X
    sc = n * U * np.ldexp(1.0, np.frexp(np.abs(A).max(1))[1])[:, None] * \
        np.ldexp(1.0, np.frexp(np.abs(X).max(0))[1])[None, :]
    assert np.all(np.abs(Y - ref) <= sc / 4)


def test_sliced_zero_rows_and_columns(L):
    rng = np.random.default_rng(3)
    n = 300
    A = rng.standard_normal((n, n))
    A = (A + A.T) / 2
    A[5, :] = 0.0
    A[:, 5] = 0.0
    X = rng.standard_normal((n, 3))
    X[:, 1] = 0.0
    Y = _apply(L, A, X)
    assert np.all(Y[5] == 0.0) and np.all(Y[:, 1] == 0.0)
    np.testing.assert_allclose(Y, A @ X, rtol=0, atol=1e-12 * np.abs(A @ X).max())


@pytest.mark.parametrize("prec", [2, 3])
def test_sliced_solver_matches_definition(L, prec):
    p = synth.config(0)
    lam_r, Xr, _ = R.lrep_definition(p["K"], p["M"], 4)
    prob = L.Problem.dense(p["K"], p["M"])
    prob.set_options(precision=prec)
    assert prob.solve(4, 4, 1e-10) == L.OK
    check(R.DenseOp(p["K"], p["M"]), prob, lam_r, 1e-10, 4, X_ref=Xr)
    prob.close()


@pytest.mark.parametrize("prec", [2, 3])
def test_sliced_solver_full_size_dense(L, prec):
    """n = 8192 with a 4-dim nullspace of K, nev 64 in windows of 16, tol
    1e-10: eigenvalues against the stored definition-route values, residuals
    re-checked on the CPU for every pair."""
    g = load_golden("config1_lambda.txt")
    p = synth.config(1)
    prob = L.Problem.dense(p["K"], p["M"])
    prob.set_nullspace(p["X0"])
    prob.set_options(precision=prec)
    assert prob.solve(64, 16, 1e-10) == L.OK
    check(R.DenseOp(p["K"], p["M"]), prob, g, 1e-10, 64)
    prob.close()


# ---------------------------------------------- tall-skinny Gram and update


def _colscale(M):
    return np.array([math.frexp(v)[1] if v > 0 else 0 for v in np.abs(M).max(axis=0)])


@pytest.mark.parametrize("n,a,b", [(70001, 40, 33), (5000, 130, 70), (300, 5, 1)])
def test_sliced_gram_error_bound(L, n, a, b):
    """G = A^T B: ragged n (many k-tiles and splits), two row tiles, three
    column groups; entries over ~20 binades."""
    import torch
    rng = np.random.default_rng(n + a + b)
    A = rng.standard_normal((n, a)) * np.exp(rng.uniform(-7, 7, (n, a)))
    B = rng.standard_normal((n, b)) * np.exp(rng.uniform(-7, 7, (n, b)))
    Ad = torch.tensor(np.ascontiguousarray(A.T), device="cuda")
    Bd = torch.tensor(np.ascontiguousarray(B.T), device="cuda")
    Gd = torch.full((b, a), np.nan, dtype=torch.float64, device="cuda")
    L.gram(Ad, Bd, Gd, sliced=True)
    torch.cuda.synchronize()
    G = Gd.cpu().numpy().T
    assert np.all(np.isfinite(G))
    ea, eb = _colscale(A), _colscale(B)
    worst = 0.0
    for i in rng.choice(a, min(a, 10), replace=False):
        for j in rng.choice(b, min(b, 6), replace=False):
            scale = n * U * 2.0 ** (ea[i] + eb[j])
            worst = max(worst, _err(G[i, j], _exact_dot(A[:, i], B[:, j])) / scale)
    assert worst <= 1.0 / 8, worst


def test_sliced_gram_and_update_exact_on_short_mantissas(L):
    import torch
    rng = np.random.default_rng(77)
    n, a, k, c = 3001, 37, 97, 45
    A = rng.integers(-2048, 2049, (n, a)).astype(np.float64) * 2.0 ** -6
    B = rng.integers(-512, 513, (n, a)).astype(np.float64)
    Gd = torch.zeros((a, a), dtype=torch.float64, device="cuda")
    L.gram(torch.tensor(A.T.copy(), device="cuda"), torch.tensor(B.T.copy(), device="cuda"),
           Gd, sliced=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Gd.cpu().numpy().T, A.T @ B)
    T = rng.integers(-1000, 1001, (n, k)).astype(np.float64) * 2.0 ** -4
    W = rng.integers(-300, 301, (k, c)).astype(np.float64)
    C0 = rng.integers(-100, 101, (n, c)).astype(np.float64)
    Cd = torch.tensor(C0.T.copy(), device="cuda")
    L.update(torch.tensor(T.T.copy(), device="cuda"), torch.tensor(W.T.copy(), device="cuda"),
             Cd, 0.5, -2.0, sliced=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Cd.cpu().numpy().T, 0.5 * C0 - 2.0 * (T @ W))


@pytest.mark.parametrize("n,k,c", [(5000, 97, 45), (20000, 384, 32), (129, 1, 3)])
def test_sliced_update_error_bound(L, n, k, c):
    """C = alpha C + beta A B with per-row scales of the tall A."""
    import torch
    rng = np.random.default_rng(n + k + c)
    A = rng.standard_normal((n, k)) * np.exp(rng.uniform(-7, 7, (n, 1)) + rng.uniform(-3, 3, (n, k)))
    B = rng.standard_normal((k, c)) * np.exp(rng.uniform(-5, 5, (k, c)))
    C0 = rng.standard_normal((n, c))
    alpha, beta = 0.75, -1.25
    Cd = torch.tensor(C0.T.copy(), device="cuda")
    L.update(torch.tensor(A.T.copy(), device="cuda"), torch.tensor(B.T.copy(), device="cuda"),
             Cd, alpha, beta, sliced=True)
    torch.cuda.synchronize()
    Cg = Cd.cpu().numpy().T
    ra = np.array([math.frexp(v)[1] if v > 0 else 0 for v in np.abs(A).max(axis=1)])
    fb = _colscale(B)
    worst = 0.0
    for i in rng.choice(n, min(n, 12), replace=False):
        for j in rng.choice(c, min(c, 6), replace=False):
            num, den = _exact_dot(A[i], B[:, j])
            exact = alpha * C0[i, j] + beta * (num / den)
            # rounding of the last fma against the exact float64 combination
            bound = abs(beta) * k * U * 2.0 ** (ra[i] + fb[j]) / 8 + 4 * U * (abs(exact) + abs(alpha * C0[i, j]))
            worst = max(worst, abs(Cg[i, j] - exact) / bound)
    assert worst <= 1.0, worst


@pytest.mark.parametrize("prec_name", ["PREC_FP64_SLICED", "PREC_MIXED_SLICED"])
def test_sliced_tall_skinny_full_size_stencil(L, prec_name):
    """The 64^3 BdG-like stencil workload with precision FP64_SLICED (the
    stencil products stay FP64, the Grams and block updates run sliced on the
    tensor cores) and MIXED_SLICED (the CG products of eq. block_GS in
    float32 arithmetic as well); same eigenvalues as the oracle's stored
    literal Alg. 2 run, residuals and biorthogonality re-checked on the
    CPU."""
    from test_gpu_solver import _stored_run
    lam_ref, _ = _stored_run("config2_oracle_run.txt")
    p = synth.config(2)
    op = R.StencilOp(p["nx"], p["ny"], p["nz"], p["h"], -0.5, p["dK"], p["dM"])
    prob = L.Problem.stencil(p["nx"], p["ny"], p["nz"], p["h"], -0.5, p["dK"], p["dM"])
    prob.set_nullspace(p["X0"])
    prob.set_options(precision=getattr(L, prec_name))
    assert prob.solve(32, 16, 1e-10) == L.OK
    lam, X, Y = check(op, prob, lam_ref, 1e-10, 32, rtol=1e-10)
    assert np.abs(p["X0"][:, 0] @ Y).max() < 1e-9
    prob.close()
