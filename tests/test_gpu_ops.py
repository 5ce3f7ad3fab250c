"""Per-step parity of the CUDA kernels with the FP64 oracle, through the
C ABI (include/lrep_ops.h).  Sizes span several tiles and a ragged tail.

Tolerances for float64 products follow the standard rounding bound: two
evaluations of a length-k dot product in different orders differ by at
most 2 * gamma_k * (|a|^T |b|), gamma_k = k u / (1 - k u), u = 2^-53.
"""
import numpy as np
import pytest

from conftest import from_dev, to_dev
from oracle import lrep_ref as R
from oracle.philox import normal_block
from paper_2506_08355_gb300 import synth

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def bound(A, B, k):
    g = k * U / (1 - k * U)
    return 2.0 * g * (np.abs(A) @ np.abs(B)) + 1e-300


@pytest.fixture(scope="module")
def L(built_lib):
    from paper_2506_08355_gb300 import lrep
    return lrep


def test_dense_apply_ragged(L):
    rng = np.random.default_rng(0)
    n, c = 1000, 37
    A = rng.standard_normal((n, n))
    K = A + A.T
    M = K @ K / n + np.eye(n)
    X = rng.standard_normal((n, c))
    p = L.Problem.dense(K, M)
    Xd = to_dev(X)
    Y = L.device_block(n, c)
    for op, mat in ((L.OP_K, K), (L.OP_M, M)):
        p.apply(op, Xd, Y)
        got = from_dev(Y)
        ref = R.DenseOp(K, M).apply("K" if op == L.OP_K else "M", X)
        assert np.all(np.abs(got - ref) <= bound(mat, X, n))
    p.close()


def test_dense_apply_split_k_sampled(L):
    """n = 8192, 16 columns (the CG product of the 8192 workload), split-K."""
    rng = np.random.default_rng(1)
    n, c = 8192, 16
    A = rng.standard_normal((n, n))
    K = (A + A.T) * 0.5
    X = rng.standard_normal((n, c))
    p = L.Problem.dense(K, K)
    Y = L.device_block(n, c)
    p.apply(L.OP_K, to_dev(X), Y)
    got = from_dev(Y)
    rows = rng.choice(n, 64, replace=False)
    ref = K[rows] @ X
    assert np.all(np.abs(got[rows] - ref) <= bound(K[rows], X, n))
    p.close()


def test_stencil_and_csr_apply(L):
    nx, ny, nz = 20, 17, 13
    s = synth.bdg_stencil(nx, ny, nz)
    op = R.StencilOp(nx, ny, nz, s["h"], -0.5, s["dK"], s["dM"])
    n = op.n
    X = np.random.default_rng(2).standard_normal((n, 19))
    ps = L.Problem.stencil(nx, ny, nz, s["h"], -0.5, s["dK"], s["dM"])
    csrK = synth.stencil_to_csr(nx, ny, nz, s["h"], -0.5, s["dK"])
    csrM = synth.stencil_to_csr(nx, ny, nz, s["h"], -0.5, s["dM"])
    pc = L.Problem.csr(n, csrK, csrM)
    Y = L.device_block(n, 19)
    for op_id, w in ((L.OP_K, "K"), (L.OP_M, "M")):
        ref = op.apply(w, X)
        scale = np.abs(op.c) * 7 * np.abs(X).max() + np.abs(op.dK).max() * np.abs(X).max()
        for prob in (ps, pc):
            prob.apply(op_id, to_dev(X), Y)
            np.testing.assert_allclose(from_dev(Y), ref, rtol=0, atol=1e-14 * scale)
    ps.close()
    pc.close()


@pytest.mark.parametrize("n,a,b", [(5000, 45, 70), (33, 3, 1), (70000, 16, 16), (4097, 80, 80)])
def test_gram(L, n, a, b):
    import torch
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, a))
    B = rng.standard_normal((n, b))
    G = torch.zeros((b, a), dtype=torch.float64, device="cuda")
    L.gram(to_dev(A), to_dev(B), G)
    torch.cuda.synchronize()
    got = G.cpu().numpy().T
    assert np.all(np.abs(got - A.T @ B) <= bound(A.T, B, n))


def test_update(L):
    import torch
    rng = np.random.default_rng(3)
    n, k, c = 3001, 45, 41
    A = rng.standard_normal((n, k))
    Bm = rng.standard_normal((k, c))
    C0 = rng.standard_normal((n, c))
    Cd = to_dev(C0)
    L.update(to_dev(A), to_dev(Bm), Cd, 0.5, -2.0)
    torch.cuda.synchronize()
    ref = 0.5 * C0 - 2.0 * (A @ Bm)
    tolm = 2.0 * bound(A, Bm, k + 1) + 4 * U * np.abs(C0)
    assert np.all(np.abs(from_dev(Cd) - ref) <= tolm)


@pytest.mark.parametrize("d", [1, 12, 37, 80, 160])
def test_small_lrep(L, d):
    import torch
    rng = np.random.default_rng(d)
    A = rng.standard_normal((d, d))
    Bq = rng.standard_normal((d, d))
    Kh = A @ A.T + 0.5 * np.eye(d)
    Mh = Bq @ Bq.T + 0.5 * np.eye(d)
    lam_r, Xr, Yr = R.small_lrep(Kh, Mh)
    lam = torch.zeros(d, dtype=torch.float64, device="cuda")
    Xh = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    Yh = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    info = L.small_lrep(to_dev(Kh), to_dev(Mh), lam, Xh, Yh)
    assert info == 0
    lg, Xg, Yg = lam.cpu().numpy(), from_dev(Xh), from_dev(Yh)
    np.testing.assert_allclose(lg, lam_r, rtol=1e-11)
    # unique up to the sign of each pair (simple spectrum)
    sg = np.sign(np.sum(Xg * Xr, axis=0))
    np.testing.assert_allclose(Xg * sg, Xr, atol=1e-9 * np.abs(Xr).max())
    np.testing.assert_allclose(Yg * sg, Yr, atol=1e-9 * np.abs(Yr).max())
    np.testing.assert_allclose(Xg.T @ Yg, np.eye(d), atol=1e-11)


@pytest.mark.parametrize("d,mult", [(40, 4), (80, 2), (24, 24)])
def test_small_lrep_degenerate(L, d, mult):
    """Repeated eigenvalues (K^ M^ with a `mult`-fold eigenvalue, and the
    fully degenerate K^ = M^ = 2 I): the eigenvalues are unique, the pairs
    inside a cluster are not; check the values, K^ X^ = Y^ Lam,
    M^ Y^ = X^ Lam and X^T Y^ = I."""
    import torch
    rng = np.random.default_rng(100 + d + mult)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    ev = np.concatenate([np.full(mult, 1.5), rng.uniform(2.0, 9.0, d - mult)])
    if mult == d:
        ev = np.full(d, 2.0)
    A = (Q * ev) @ Q.T          # K^ = M^ = A: eigenvalues of K^ M^ are ev^2
    lam = torch.zeros(d, dtype=torch.float64, device="cuda")
    Xh = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    Yh = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    info = L.small_lrep(to_dev(A), to_dev(A), lam, Xh, Yh)
    assert info == 0
    lg, Xg, Yg = lam.cpu().numpy(), from_dev(Xh), from_dev(Yh)
    np.testing.assert_allclose(lg, np.sort(ev), rtol=1e-12)
    sc = np.abs(A).max() * max(1.0, np.abs(Xg).max())
    np.testing.assert_allclose(A @ Xg, Yg * lg, atol=1e-11 * sc)
    np.testing.assert_allclose(A @ Yg, Xg * lg, atol=1e-11 * sc)
    np.testing.assert_allclose(Xg.T @ Yg, np.eye(d), atol=1e-11)


def test_small_lrep_not_spd(L):
    import torch
    d = 6
    Kh = np.diag([1.0, 2.0, -1.0, 3.0, 4.0, 5.0])
    lam = torch.zeros(d, dtype=torch.float64, device="cuda")
    Xh = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    Yh = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    assert L.small_lrep(to_dev(Kh), to_dev(np.eye(d)), lam, Xh, Yh) == 1
    assert L.small_lrep(to_dev(np.eye(d)), to_dev(Kh), lam, Xh, Yh) == 2


def test_biorth_matches_alg1(L):
    """The biorthogonal pair is unique (LU of W^T Z with the Alg. 1
    normalisation), so GPU and the literal Alg. 1 agree column by column,
    including which pair is discarded."""
    rng = np.random.default_rng(5)
    n, m = 3000, 24
    W = rng.standard_normal((n, m))
    Z = W + 0.5 * rng.standard_normal((n, m))
    W[:, 7] = W[:, 2] - 0.5 * W[:, 5]
    Z[:, 7] = Z[:, 2] - 0.5 * Z[:, 5]   # pair 7 in the span of pairs 2, 5
    Pr, Qr, kept = R.mgs_biorth(W, Z)
    P = L.device_block(n, m)
    Q = L.device_block(n, m)
    k = L.biorth(to_dev(W), to_dev(Z), P, Q)
    assert k == len(kept) == m - 1
    Pg, Qg = from_dev(P)[:, :k], from_dev(Q)[:, :k]
    np.testing.assert_allclose(Pg, Pr, atol=1e-9 * np.abs(Pr).max())
    np.testing.assert_allclose(Qg, Qr, atol=1e-9 * np.abs(Qr).max())
    np.testing.assert_allclose(Pg.T @ Qg, np.eye(k), atol=1e-12)


def test_residuals(L):
    import torch
    rng = np.random.default_rng(6)
    n, w = 2500, 9
    X, Y = rng.standard_normal((n, w)), rng.standard_normal((n, w))
    KX, MY = rng.standard_normal((n, w)), rng.standard_normal((n, w))
    lam = rng.uniform(0.1, 2.0, w)
    eps = torch.zeros(w, dtype=torch.float64, device="cuda")
    L.residuals(to_dev(X), to_dev(Y), to_dev(KX), to_dev(MY),
                torch.from_numpy(lam).cuda(), eps)

    class Fixed:
        def apply(self, which, Z):
            return KX if which == "K" else MY
    ref = R.residuals(Fixed(), X, Y, lam)
    np.testing.assert_allclose(eps.cpu().numpy(), ref, rtol=1e-13)


def test_philox_normals(L):
    import torch
    n, c = 1001, 7
    out = L.device_block(n, c)
    L.philox_normal(n, c, 0x123456789ABCDEF, 1, out)
    torch.cuda.synchronize()
    ref = normal_block(n, c, 0x123456789ABCDEF, 1)
    np.testing.assert_allclose(from_dev(out), ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("n,c", [(1000, 16), (1000, 1), (777, 37), (4096, 32), (200, 4),
                                 (8192, 16), (12000, 32), (12000, 17), (5000, 64)])
def test_bf16x3_tensor_core_product(L, n, c):
    """Mixed-precision CG product (tcgen05, bf16 hi/lo split, fp32
    accumulation) against the float64 product.  Error model: dropping the
    lo*lo term and rounding lo leave ~2^-16 relative per operand, fp32
    accumulation adds ~k 2^-24; bound 1e-4 of |A||X| with margin.  Shapes
    with ragged row tiles, k-tiles and column counts (N padded to 16)."""
    rng = np.random.default_rng(n + c)
    A = rng.standard_normal((n, n))
    K = (A + A.T) * 0.5
    del A
    M = (K @ K / n + np.eye(n)) if n <= 4096 else (0.3 * K + 2.0 * np.eye(n))
    X = rng.standard_normal((n, c))
    p = L.Problem.dense(K, M)
    p.set_options(precision=L.PREC_MIXED_BF16X3)
    Y = L.device_block(n, c)
    for op, mat in ((L.OP_K, K), (L.OP_M, M)):
        p.apply(op, to_dev(X), Y, cg=True)
        got = from_dev(Y)
        ref = mat @ X
        scale = np.abs(mat) @ np.abs(X)
        err = np.abs(got - ref) / scale
        assert err.max() < 1e-4, err.max()
        # and it is not the float64 path: the error is visibly non-zero
        assert err.max() > 1e-12
    p.close()


@pytest.mark.parametrize("prec_name", ["PREC_FP64", "PREC_FP64_SLICED"])
def test_cg_matches_oracle_columnwise(L, prec_name):
    """The CG of eq. block_GS (lrep_op_cg: the solver's cg_init / cg_alpha /
    cg_update / cg_pdir kernels and its CG operator) against the oracle's
    cg, column by column: at fixed iteration counts with no stopping, and
    with the paper's tolerance 1e-2 (per-column stops, same iteration
    count).  A zero right-hand side stays inactive on both sides.  Float64
    products: the iterates agree to rounding amplified by the few steps
    (bound 1e-11 relative to the column's norm)."""
    from oracle import lrep_ref as R
    n, c = 3000, 12
    rng = np.random.default_rng(77)
    p = synth.haar_dense(n, seed=77)
    K, M = p["K"], p["M"]
    B = rng.standard_normal((n, c))
    B[:, 5] = 0.0
    prob = L.Problem.dense(K, M)
    prob.set_options(precision=getattr(L, prec_name))
    Bd = to_dev(B)
    Xd = L.device_block(n, c)
    for op, mat in ((L.OP_K, K), (L.OP_M, M)):
        for tol, maxit in ((0.0, 1), (0.0, 5), (0.0, 12), (1e-2, 60)):
            its = prob.cg(op, Bd, Xd, tol, maxit)
            X = from_dev(Xd)
            Xr, its_r = R.cg(lambda Z: mat @ Z, B, tol, maxit)
            assert its == its_r, (op, tol, maxit, its, its_r)
            scale = np.maximum(np.linalg.norm(Xr, axis=0), 1e-300)
            err = np.linalg.norm(X - Xr, axis=0) / scale
            assert err.max() < 1e-11, (op, tol, maxit, err.max())
            assert np.all(X[:, 5] == 0.0)
    prob.close()



@pytest.mark.parametrize("prec_name", ["PREC_MIXED_BF16X3", "PREC_MIXED_SLICED"])
@pytest.mark.parametrize("n,c", [(3000, 12), (8192, 32)])
def test_cg_mixed_matches_oracle_columnwise(L, prec_name, n, c):
    """The CG of eq. block_GS on the bf16 hi/lo tensor-core operator
    (lrep_op_cg: each step is the tensor-core product plus the one-launch
    CG step kernel, which sums the product's split-K partials, updates x, r
    and p and writes the next product's bf16 operand) against the oracle's
    float64 cg, column by column.  The products carry ~2^-16 relative error,
    which moves the iterates by ~1e-5 of the column's norm over 12 steps
    (a numpy model of the split gives 9e-6), so the bound is 1e-4; with the
    paper's tolerance 1e-2 the iteration counts agree within one and every
    column's float64 residual meets the tolerance.  n = 3000: 24 row tiles
    with a ragged tail; n = 8192: a 4-way split-K sum."""
    from oracle import lrep_ref as R
    rng = np.random.default_rng(78)
    p = synth.haar_dense(n, seed=78)
    K, M = p["K"], p["M"]
    B = rng.standard_normal((n, c))
    B[:, 5] = 0.0
    prob = L.Problem.dense(K, M)
    prob.set_options(precision=getattr(L, prec_name))
    Bd = to_dev(B)
    Xd = L.device_block(n, c)
    bn = np.maximum(np.linalg.norm(B, axis=0), 1e-300)
    for op, mat in ((L.OP_K, K), (L.OP_M, M)):
        for tol, maxit in ((0.0, 1), (0.0, 5), (0.0, 12), (1e-2, 60)):
            its = prob.cg(op, Bd, Xd, tol, maxit)
            X = from_dev(Xd)
            Xr, its_r = R.cg(lambda Z: mat @ Z, B, tol, maxit)
            assert np.all(X[:, 5] == 0.0)
            if tol == 0.0:
                assert its == its_r == maxit, (op, maxit, its, its_r)
                scale = np.maximum(np.linalg.norm(Xr, axis=0), 1e-300)
                err = np.linalg.norm(X - Xr, axis=0) / scale
                assert err.max() < 1e-4, (op, maxit, err.max())
            else:
                assert abs(its - its_r) <= 1, (op, its, its_r)
                res = np.linalg.norm(B - mat @ X, axis=0) / bn
                assert res.max() <= 1.01e-2, (op, res.max())
    prob.close()


@pytest.mark.parametrize("dims", [(17, 9, 5), (64, 64, 64)])
def test_stencil_float32_cg_product(L, dims):
    """The stencil's CG product under the mixed precision (float32 sums,
    float64 loads and stores) against the float64 product: error bounded by
    ~2^-23 of |coef| |Lap| |X| + |d| |X| (bound 1e-6 of that scale), and
    visibly not the float64 path."""
    nx, ny, nz = dims
    s = synth.bdg_stencil(nx, ny, nz)
    n = s["n"]
    rng = np.random.default_rng(nx)
    X = rng.standard_normal((n, 5))
    p = L.Problem.stencil(nx, ny, nz, s["h"], -0.5, s["dK"], s["dM"])
    p.set_options(precision=L.PREC_MIXED_BF16X3)
    op = R.StencilOp(nx, ny, nz, s["h"], -0.5, s["dK"], s["dM"])
    absop = R.StencilOp(nx, ny, nz, s["h"], 0.5, np.abs(s["dK"]) + 6.0 / s["h"] ** 2,
                        np.abs(s["dM"]) + 6.0 / s["h"] ** 2)
    Y = L.device_block(n, 5)
    for which, name in ((L.OP_K, "K"), (L.OP_M, "M")):
        p.apply(which, to_dev(X), Y, cg=True)
        got = from_dev(Y)
        ref = op.apply(name, X)
        scale = absop.apply(name, np.abs(X))
        err = (np.abs(got - ref) / scale).max()
        assert err < 1e-6, err
        assert err > 1e-12
    p.close()
