"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  None of them re-types an oracle
formula: they use printed values (tests/golden), closed forms, invariants,
brute force on tiny inputs, or an independent factorisation.
"""
import math

import numpy as np
import pytest
from scipy.linalg import eigh_tridiagonal, hilbert

from conftest import load_golden
from oracle import lrep_ref as R
from oracle.philox import normal_block, philox4x32_10
from paper_2506_08355_gb300 import synth


# ---------------------------------------------------------------- Philox


def test_philox_known_answers():
    """Random123 known-answer vectors for philox4x32-10."""
    cases = [
        ([0, 0, 0, 0], [0, 0],
         [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2,
         [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
         [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        assert [int(v) for v in philox4x32_10(ctr, key)] == want


def test_philox_normals_moments():
    z = normal_block(20000, 3, seed=7, stream=1)
    assert z.shape == (20000, 3)
    assert abs(z.mean()) < 0.02
    assert abs(z.std() - 1.0) < 0.02
    # streams and seeds give different draws
    assert not np.allclose(z, normal_block(20000, 3, seed=7, stream=0))


# ---------------------------------------------------- R1: the definition


def test_definition_example1_closed_form_and_table2():
    """Example 1: K = M = T(0); lam_l = 4 sin^2(pi l / (2(n+1))) (Sec. 4.1)."""
    n = 1000
    T = synth.tridiag_T(n, 0.0)
    lam, X, Y = R.lrep_definition(T, T, 10)
    k = np.arange(1, 11)
    exact = 4.0 * np.sin(np.pi * k / (2.0 * (n + 1))) ** 2
    g = load_golden("table2_example1.txt")
    # the golden exact column is the closed form (checks the transcription)
    np.testing.assert_allclose(g[:, 1], exact, rtol=1e-15)
    # SVD route: absolute accuracy ~ eps * ||H|| (||H|| = 4)
    assert np.max(np.abs(lam - exact)) < 1e-13
    # vectors x = y = sin(j l pi/(n+1)) up to scale: x^T y = 1 fixes scale
    j = np.arange(1, n + 1)
    for c in range(3):
        s = np.sin(j * (c + 1) * np.pi / (n + 1))
        s = s / math.sqrt(s @ s)
        assert abs(abs(X[:, c] @ s) - 1.0) < 1e-9
        np.testing.assert_allclose(X[:, c], Y[:, c], atol=1e-9)


def test_definition_example2_table3():
    """Example 2: K = T(-1) singular, M = T(0); Table 3 Advanpix column."""
    n = 1000
    K = synth.tridiag_T(n, -1.0)
    M = synth.tridiag_T(n, 0.0)
    lam, X, Y = R.lrep_definition(K, M, 10, r=1)
    g = load_golden("table3_example2.txt")
    # 13 printed digits; absolute accuracy of the SVD route ~ eps * 4
    np.testing.assert_allclose(lam, g[:, 1], rtol=2e-11)


def test_definition_commuting_spectra():
    """Q1 = Q2 = Q: K M = Q diag(k m) Q^T, so lam_i = sqrt(k_i m_i)."""
    p = synth.haar_dense(60, seed=11, commuting=True)
    lam, X, Y = R.lrep_definition(p["K"], p["M"], 8)
    ref = np.sort(np.sqrt(p["k"] * p["m"]))[:8]
    np.testing.assert_allclose(lam, ref, rtol=1e-12)
    # x = Q e_i (m_i/k_i)^{1/4}, y = Q e_i (k_i/m_i)^{1/4}
    order = np.argsort(np.sqrt(p["k"] * p["m"]))[:8]
    for c, i in enumerate(order):
        q = p["Q1"][:, i]
        xs = q * (p["m"][i] / p["k"][i]) ** 0.25
        ys = q * (p["k"][i] / p["m"][i]) ** 0.25
        sgn = np.sign(X[:, c] @ xs)
        np.testing.assert_allclose(sgn * X[:, c], xs, atol=1e-10)
        np.testing.assert_allclose(sgn * Y[:, c], ys, atol=1e-10)


def test_definition_bruteforce_eig_of_H_and_pairing():
    """Brute force: eigenvalues of the 2n x 2n H come in pairs +-lam
    (Lemma eigReal (iii)); the positive ones are R1's."""
    p = synth.haar_dense(9, seed=3, n_zero_k=1)
    K, M = p["K"], p["M"]
    H = np.block([[np.zeros((9, 9)), K], [M, np.zeros((9, 9))]])
    ev = np.sort(np.linalg.eigvals(H).real)
    lam, X, Y = R.lrep_definition(K, M, 8, r=1)
    pos = np.sort(ev[ev > 1e-6])
    neg = np.sort(-ev[ev < -1e-6])
    np.testing.assert_allclose(pos, lam, rtol=1e-9)
    np.testing.assert_allclose(neg, lam, rtol=1e-9)
    # eigen-equations and biorthogonality (Lemma eigPairing)
    np.testing.assert_allclose(K @ X, Y * lam, atol=1e-12)
    np.testing.assert_allclose(M @ Y, X * lam, atol=1e-12)
    np.testing.assert_allclose(X.T @ Y, np.eye(8), atol=1e-12)
    # [-y; x] belongs to -lam
    xi = np.concatenate([-Y[:, 0], X[:, 0]])
    np.testing.assert_allclose(H @ xi, -lam[0] * xi, atol=1e-12)


def test_definition_values_only_route():
    p = synth.haar_dense(50, seed=9, n_zero_k=2)
    lam, X, Y = R.lrep_definition(p["K"], p["M"], 10, r=2)
    FK = p["Q1"] * np.sqrt(p["k"])[None, :]
    FM = p["Q2"] * np.sqrt(p["m"])[None, :]
    np.testing.assert_allclose(R.lrep_definition_values(FK, FM, 10, r=2), lam, rtol=1e-12)


def test_trace_minimisation_principle():
    """Thm. minimization principles: sum of the k smallest lam equals
    1/2 tr(U^T K U + V^T M V) at the eigenvectors and is a lower bound for
    other biorthogonal pairs (U^T V = I) biorthogonal to V0."""
    p = synth.haar_dense(40, seed=8)
    K, M = p["K"], p["M"]
    lam, X, Y = R.lrep_definition(K, M, 5)
    val = 0.5 * np.trace(X.T @ K @ X + Y.T @ M @ Y)
    assert abs(val - lam.sum()) < 1e-12 * lam.sum()
    rng = np.random.default_rng(1)
    for _ in range(5):
        U = X + 0.05 * rng.standard_normal(X.shape)
        V = Y + 0.05 * rng.standard_normal(Y.shape)
        S = U.T @ V
        V = V @ np.linalg.inv(S)  # now U^T V = I
        tr = 0.5 * np.trace(U.T @ K @ U + V.T @ M @ V)
        assert tr > lam.sum()


def test_residual_definition():
    """eq. tol: zero at exact pairs; equal to the hand value for a
    perturbed pair of a 2 x 2 diagonal problem."""
    K = np.diag([4.0, 9.0])
    M = np.eye(2)
    op = R.DenseOp(K, M)
    # exact pair: lam = 2, x = e1/sqrt2 ... K x = 4 x = lam y -> y = 2 x
    x = np.array([[1.0], [0.0]]) / math.sqrt(2.0)
    y = 2.0 * x
    assert R.residuals(op, x, y, np.array([2.0]))[0] < 1e-16
    # perturbed: lam = 1 -> Kx - y = (4 - 2)/sqrt2 e1, My - x = (2-1)/sqrt2 e1
    e = R.residuals(op, x, y, np.array([1.0]))[0]
    want = math.sqrt(2.0 + 0.5) / (2.0 * math.sqrt(0.5 + 2.0))
    assert abs(e - want) < 1e-15


# ------------------------------------------------------------ Alg. 1


def _lauchli(n, mu):
    L = np.zeros((n, n - 1))
    L[0, :] = 1.0
    L[1:, :] = mu * np.eye(n - 1)
    return L


def test_mgs_cgs_table1():
    """Table 1: Hilbert / Lauchli (mu = 1e-3) inputs; condition numbers
    to 3 digits and biorthogonality losses within 10x of the printed ones
    (the bits depend on the rounding order)."""
    g = load_golden("table1_biorth.txt")
    for row in g:
        n = int(row[0])
        m = n // 2
        X = hilbert(n)[:, :m]
        Y = _lauchli(n, 1e-3)[:, :m]
        assert abs(np.linalg.cond(X) / row[1] - 1) < 0.01
        assert abs(np.linalg.cond(Y) / row[2] - 1) < 0.01
        P, Q, kept = R.mgs_biorth(X, Y, tau=0.0)
        assert len(kept) == m
        mgs = np.linalg.norm(P.T @ Q - np.eye(m), 2)
        P2, Q2 = R.cgs_biorth(X, Y)
        cgs = np.linalg.norm(P2.T @ Q2 - np.eye(m), 2)
        assert row[5] / 10 < mgs < row[5] * 10, (n, mgs)
        if n <= 12:
            assert row[4] / 10 < cgs < row[4] * 10, (n, cgs)
        else:
            assert cgs > 1.0  # CGS has lost biorthogonality completely


def _lu_nopivot(A):
    """Doolittle LU without pivoting, for the identity check below."""
    m = A.shape[0]
    L = np.eye(m)
    U = A.astype(float).copy()
    for k in range(m):
        for i in range(k + 1, m):
            L[i, k] = U[i, k] / U[k, k]
            U[i, :] -= L[i, k] * U[k, :]
    return L, U


def test_mgs_biorth_equals_lu_construction():
    """Exact-arithmetic identity: MGS-Biorth gives P = X R^-1, Q = Y S^-1
    with X^T Y = R^T S (R, S upper triangular, r_ll = sign(u_ll) sqrt|u_ll|,
    s_ll = sqrt|u_ll|), i.e. the LU factorisation of X^T Y."""
    rng = np.random.default_rng(2)
    n, m = 50, 7
    X = rng.standard_normal((n, m))
    Y = X + 0.3 * rng.standard_normal((n, m))
    P, Q, kept = R.mgs_biorth(X, Y)
    assert kept == list(range(m))
    L, U = _lu_nopivot(X.T @ Y)
    u = np.diag(U)
    r = np.sign(u) * np.sqrt(np.abs(u))
    Rm = np.diag(r) @ L.T
    Sm = np.diag(1.0 / r) @ U
    np.testing.assert_allclose(P, X @ np.linalg.inv(Rm), atol=1e-11)
    np.testing.assert_allclose(Q, Y @ np.linalg.inv(Sm), atol=1e-11)
    np.testing.assert_allclose(P.T @ Q, np.eye(m), atol=1e-13)


def test_mgs_discard_rule():
    """Remark after Alg. 1: a pair whose running eta vanishes is dropped."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((30, 4))
    Y = rng.standard_normal((30, 4))
    X[:, 2] = X[:, 0] + 2.0 * X[:, 1]   # dependent: p_3 -> 0 after projection
    P, Q, kept = R.mgs_biorth(X, Y)
    assert kept == [0, 1, 3]
    np.testing.assert_allclose(P.T @ Q, np.eye(3), atol=1e-12)


# ------------------------------------------------------- small LREP


def test_small_lrep_bruteforce():
    """eq. small_eigen: the d positive eigenvalues of [[0,K^],[M^,0]]
    (brute-force eigvals) with K^ X^ = Y^ L, M^ Y^ = X^ L, X^T Y^ = I."""
    rng = np.random.default_rng(5)
    d = 12
    A = rng.standard_normal((d, d))
    B = rng.standard_normal((d, d))
    Kh = A @ A.T + 0.1 * np.eye(d)
    Mh = B @ B.T + 0.1 * np.eye(d)
    lam, Xh, Yh = R.small_lrep(Kh, Mh)
    H = np.block([[np.zeros((d, d)), Kh], [Mh, np.zeros((d, d))]])
    ev = np.sort(np.linalg.eigvals(H).real)
    np.testing.assert_allclose(lam, ev[d:], rtol=1e-10)
    np.testing.assert_allclose(Kh @ Xh, Yh * lam, atol=1e-10)
    np.testing.assert_allclose(Mh @ Yh, Xh * lam, atol=1e-10)
    np.testing.assert_allclose(Xh.T @ Yh, np.eye(d), atol=1e-12)


def test_small_lrep_not_spd_raises():
    Kh = np.diag([1.0, -1.0])
    with pytest.raises(np.linalg.LinAlgError):
        R.small_lrep(Kh, np.eye(2))


# ------------------------------------------------------ nullspace, CG


def test_nullspace_example2_closed_form():
    """Example 2: x0 = 1, M y0 = x0 has y0_l = l (n - l + 1) / 2; after
    eq. V0_basis X0^T Y0 = 1."""
    n = 200
    K = synth.tridiag_T(n, -1.0)
    M = synth.tridiag_T(n, 0.0)
    class MatFree:  # not a DenseOp: setup_nullspace takes its CG route
        def __init__(self):
            self.n = n

        def apply(self, which, Z):
            return (K if which == "K" else M) @ Z

    X0, Y0 = R.setup_nullspace(MatFree(), np.ones((n, 1)))
    l = np.arange(1, n + 1)
    y = l * (n - l + 1) / 2.0
    y = y / math.sqrt(np.ones(n) @ y)
    np.testing.assert_allclose(Y0[:, 0], y, rtol=1e-9)
    assert abs(X0[:, 0] @ Y0[:, 0] - 1.0) < 1e-13
    np.testing.assert_allclose(K @ X0, 0.0, atol=1e-12)


def test_cg_reaches_tolerance():
    """CG per column: relative residual below tol, or maxit reached."""
    n = 100
    M = synth.tridiag_T(n, 0.0) + 0.5 * np.eye(n)
    B = np.random.default_rng(0).standard_normal((n, 3))
    X, it = R.cg(lambda Z: M @ Z, B, 1e-10, 500)
    assert it <= n + 5
    np.testing.assert_allclose(M @ X, B, atol=1e-8)
    X2, it2 = R.cg(lambda Z: M @ Z, B, 1e-2, 3)
    assert it2 == 3


# ------------------------------------------------------- operators


def test_stencil_separable_spectrum_and_null_vector():
    """BdG-like stencil with g = 0 and d_M = d_K + c: K is a Kronecker
    sum of 1-D operators (eigenvalues from a tridiagonal eigensolver) with
    null vector phi, and lam(H) = sqrt(kappa (kappa + c))."""
    nx, c = 12, 50.0
    p = synth.bdg_stencil(nx, g=0.0, shift_c=c)
    op = R.StencilOp(nx, nx, nx, p["h"], -0.5, p["dK"], p["dM"])
    Kphi = op.apply("K", p["phi"])
    assert np.linalg.norm(Kphi) < 1e-10 * (6 / p["h"] ** 2)
    h = p["h"]
    ev1 = []
    for v in p["v1d"]:
        w = eigh_tridiagonal(1.0 / h ** 2 + v, np.full(nx - 1, -0.5 / h ** 2),
                             eigvals_only=True)
        ev1.append(w)
    kap = (ev1[2][:, None, None] + ev1[1][None, :, None]
           + ev1[0][None, None, :]).reshape(-1)
    kap = np.sort(kap)
    assert abs(kap[0]) < 1e-9 * kap[-1]
    Kd = op.apply("K", np.eye(op.n))
    np.testing.assert_allclose(np.linalg.eigvalsh(Kd), kap, atol=1e-8 * kap[-1])
    lam = np.sqrt(kap[1:] * (kap[1:] + c))
    got, X, Y = R.lrep_definition(Kd, op.apply("M", np.eye(op.n)), 6, r=1)
    np.testing.assert_allclose(got, lam[:6], rtol=1e-9)


def test_stencil_matches_csr():
    nx, ny, nz = 5, 4, 3
    p = synth.bdg_stencil(nx, ny, nz)
    op = R.StencilOp(nx, ny, nz, p["h"], -0.5, p["dK"], p["dM"])
    csr = R.CsrOp(op.n, synth.stencil_to_csr(nx, ny, nz, p["h"], -0.5, p["dK"]),
                  synth.stencil_to_csr(nx, ny, nz, p["h"], -0.5, p["dM"]))
    Z = np.random.default_rng(0).standard_normal((op.n, 3))
    for w in ("K", "M"):
        np.testing.assert_allclose(op.apply(w, Z), csr.apply(w, Z), rtol=1e-13,
                                   atol=1e-9)


# ------------------------------------------------------- R2: Alg. 2


def _check_solution(op, res, lam_ref, tol, nev):
    assert res.converged and res.nconv == nev
    np.testing.assert_allclose(res.lam, lam_ref, rtol=1e-10)
    assert R.residuals(op, res.X, res.Y, res.lam).max() < tol
    np.testing.assert_allclose(res.X.T @ res.Y, np.eye(nev), atol=1e-12)


def test_bosp_config0_vs_definition():
    p = synth.config(0)
    op = R.DenseOp(p["K"], p["M"])
    lam, X, Y = R.lrep_definition(p["K"], p["M"], 4)
    res = R.bosp(op, 4, 4, 1e-10)
    _check_solution(op, res, lam, 1e-10, 4)
    # simple eigenvalues: vectors agree (sign fixed) to ~ tol / gap
    np.testing.assert_allclose(res.X, X, atol=1e-7)
    np.testing.assert_allclose(res.Y, Y, atol=1e-7)


def test_bosp_example1_table2():
    """Example 1 at the paper's size; Table 2 reports eps_k <= 6.3e-13."""
    n = 1000
    T = synth.tridiag_T(n, 0.0)
    op = R.DenseOp(T, T)
    g = load_golden("table2_example1.txt")
    res = R.bosp(op, 10, 10, 1e-10)
    assert res.converged
    np.testing.assert_allclose(res.lam, g[:, 1], rtol=2e-12)


def test_bosp_example2_table3():
    """Example 2 (zero eigenvalue deflated through V0); Table 3."""
    n = 1000
    K = synth.tridiag_T(n, -1.0)
    M = synth.tridiag_T(n, 0.0)
    op = R.DenseOp(K, M)
    g = load_golden("table3_example2.txt")
    res = R.bosp(op, 10, 10, 1e-10, X0=np.ones((n, 1)))
    assert res.converged
    np.testing.assert_allclose(res.lam, g[:, 1], rtol=2e-11)


def test_bosp_moving_window_with_nullspace():
    """Batching + moving (Sec. 3.3): nev = 40 in batches of nb = 8 with a
    2-dim nullspace of K; every locked pair is a true eigenpair."""
    p = synth.haar_dense(500, seed=5, n_zero_k=2)
    op = R.DenseOp(p["K"], p["M"])
    lam, X, Y = R.lrep_definition(p["K"], p["M"], 40, r=2)
    res = R.bosp(op, 40, 8, 1e-10, X0=p["X0"])
    _check_solution(op, res, lam, 1e-10, 40)
    # deflated against V0: X^T Y0 = 0 (Lemma generalized nullspace (iii))
    assert np.abs(p["X0"].T @ res.Y).max() < 1e-10


def test_bosp_stencil_separable():
    """Stencil workload with the exact separable spectrum (g = 0)."""
    nx, c = 10, 40.0
    p = synth.bdg_stencil(nx, g=0.0, shift_c=c)
    op = R.StencilOp(nx, nx, nx, p["h"], -0.5, p["dK"], p["dM"])
    Kd = op.apply("K", np.eye(op.n))
    kap = np.sort(np.linalg.eigvalsh(Kd))[1:]
    lam = np.sqrt(kap * (kap + c))[:8]
    res = R.bosp(op, 8, 4, 1e-10, X0=p["phi"][:, None])
    _check_solution(op, res, lam, 1e-10, 8)


def test_nullspace_definition_recovers_chosen_kernel():
    """K = Q diag(k) Q^T with k_0..k_{r-1} = 0: the definition returns a
    basis of span(Q[:, :r]) (same orthogonal projector) and nothing else;
    with no zero k it returns an empty basis; a zero matrix is all kernel."""
    rng = np.random.default_rng(11)
    n, r = 60, 3
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = rng.uniform(0.5, 10.0, n)
    k[:r] = 0.0
    K = (Q * k) @ Q.T
    X0, w = R.nullspace_definition(K, 1e-10)
    assert X0.shape == (n, r)
    np.testing.assert_allclose(X0 @ X0.T, Q[:, :r] @ Q[:, :r].T, atol=1e-12)
    np.testing.assert_allclose(np.sort(w)[r:], np.sort(k[r:]), rtol=1e-12)
    k[:r] = 1e-3  # smallest eigenvalue 1e-4 of ||K||: not a kernel at tol 1e-10
    X1, _ = R.nullspace_definition((Q * k) @ Q.T, 1e-10)
    assert X1.shape == (n, 0)
    X2, _ = R.nullspace_definition(np.zeros((5, 5)), 1e-10)
    assert X2.shape == (5, 5)


def test_generalized_definition_pins():
    """Remark on the generalized LREP: (i) B = beta I scales the spectrum by
    1/beta and the vectors by beta^-1/2; (ii) the positive eigenvalues of
    the pencil ([[0, K], [M, 0]], diag(B, B)) by a general eigensolver;
    (iii) K X = B Y Lam, M Y = B X Lam, X^T B Y = I."""
    import scipy.linalg as sla
    rng = np.random.default_rng(21)
    n, nev = 14, 5
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    K = (Q1 * rng.uniform(0.5, 10, n)) @ Q1.T
    M = (Q2 * rng.uniform(0.5, 10, n)) @ Q2.T
    lam, X, Y = R.lrep_definition(K, M, nev)
    beta = 2.5
    lb, Xb, Yb = R.lrep_definition_gen(K, M, beta * np.eye(n), nev)
    np.testing.assert_allclose(lb, lam / beta, rtol=1e-12)
    np.testing.assert_allclose(Xb, X / np.sqrt(beta), atol=1e-10)
    A = rng.standard_normal((n, n))
    Bm = A @ A.T + n * np.eye(n)
    lg, Xg, Yg = R.lrep_definition_gen(K, M, Bm, nev)
    H = np.block([[np.zeros((n, n)), K], [M, np.zeros((n, n))]])
    Bb = np.block([[Bm, np.zeros((n, n))], [np.zeros((n, n)), Bm]])
    ev = sla.eigvals(H, Bb)
    pos = np.sort(ev.real[ev.real > 0])[:nev]
    np.testing.assert_allclose(lg, pos, rtol=1e-9)
    np.testing.assert_allclose(K @ Xg, Bm @ Yg * lg, atol=1e-9)
    np.testing.assert_allclose(M @ Yg, Bm @ Xg * lg, atol=1e-9)
    np.testing.assert_allclose(Xg.T @ Bm @ Yg, np.eye(nev), atol=1e-10)


def test_bosp_generalized_vs_definition():
    """Alg. 2 in the B-inner product (Remark on the generalized LREP)
    against the definition route through B = L L^T: simple window, moving
    window, and a singular K deflated through V0 (M Y0 = B X0)."""
    rng = np.random.default_rng(31)
    for n, nev, nb, r in ((120, 4, 4, 0), (300, 12, 4, 0), (200, 6, 3, 2)):
        Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
        Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
        k = rng.uniform(0.5, 10, n)
        k[:r] = 0.0
        K = (Q1 * k) @ Q1.T
        M = (Q2 * rng.uniform(0.5, 10, n)) @ Q2.T
        Q3, _ = np.linalg.qr(rng.standard_normal((n, n)))
        Bm = (Q3 * rng.uniform(0.5, 2.0, n)) @ Q3.T
        op = R.DenseOp(K, M, Bm)
        lam_d, Xd, Yd = R.lrep_definition_gen(K, M, Bm, nev, r)
        res = R.bosp(op, nev, nb, 1e-10, X0=Q1[:, :r] if r else None)
        assert res.converged and res.nconv == nev
        np.testing.assert_allclose(res.lam, lam_d, rtol=1e-10)
        assert R.residuals(op, res.X, res.Y, res.lam).max() < 1e-10
        np.testing.assert_allclose(res.X.T @ Bm @ res.Y, np.eye(nev), atol=1e-10)
        np.testing.assert_allclose(np.abs(res.X), np.abs(Xd), atol=1e-6)
        if r:
            assert np.abs(Q1[:, :r].T @ Bm @ res.Y).max() < 1e-9
