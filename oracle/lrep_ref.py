"""FP64 CPU oracle of the BOSP hot path (test infrastructure; see package doc).

Notation follows the paper: H = [[0, K], [M, 0]] acting on xi = [y; x] with
K = A - B symmetric positive semi-definite and M = A + B symmetric positive
definite (eq. xy_algebra); eigenpairs satisfy K x = lam y, M y = lam x,
x^T y = 1.

Routes
  R1  ``lrep_definition``: the plain definition by factorisations and one
      SVD (dense, small n).  Exact up to rounding order.
  R2  ``bosp``: a literal Alg. 2 (BOSP) with Alg. 1 (MGS-Biorth), eq. hat_H,
      the small LREP, eq. hat_pq, eq. block_GS with CG, eq. update_W/Z and
      the batching/moving window of Section 3.3.

Readings of passages that are silent or ambiguous (each listed in the
design notes):
  * small LREP (Section 3.3 cost item 2: "two Cholesky factorizations and
    one SVD"): K^ = L1 L1^T, M^ = L2 L2^T, G = L1^T L2 = W S V^T,
    X^ = L2 V S^-1/2, Y^ = L1 W S^-1/2, lam = S ascending.
  * discard rule (Remark after Alg. 1): "s_ll quite close to zero" is
    measured against the scale of the pair as it entered the
    biorthogonalisation: drop when |eta| <= tau * ||x_l|| ||y_l|| (eta not
    finite also drops), tau = 1e-10.  For W/Z the entering pair is the CG
    output before eq. update_W/Z, for P^/Q^ the vectors X^_j - E_j,
    Y^_j - E_j before the projector of eq. hat_pq.  (A test against the
    running p, q cannot see a pair that the projection reduced to rounding
    noise: noise keeps an O(1) cosine.)
  * CG (after eq. block_GS): per column, zero start, stop when
    ||r|| <= tol ||b|| (tol 1e-2) or after 20 iterations, no preconditioner.
  * KW = rhs with singular K: rhs is first projected orthogonally off
    span(X0) (range(K) is the orthogonal complement of N(K)).
  * ngs (never given) = 1.
  * window: X holds w = s*nb columns when nb < nev (moving, s = 3) and
    w = nev when nb >= nev (Alg. 2 as printed); converged = leading prefix
    with eps_i < tol; when that prefix reaches 2*nb and more pairs are
    wanted, lock those 2*nb and the new window is Ritz pairs 2nb..2nb+w-1
    of the same projected problem.
  * E in eq. hat_pq: column j of U's X block, the previous iterate of Ritz
    pair j (zero if U's X block has fewer than j+1 columns); the projector
    uses every Ritz pair from 0 to the end of the window.
  * Ritz pair signs: X^_j - E_j in eq. hat_pq is the step between
    consecutive iterates only if pair j keeps the sign of its previous
    iterate, so each pair j < (width of U's X block) is scaled by -1 when
    X^[j, j] < 0.  Without this the O(1) difference cancels to an O(step)
    direction and biorthogonality P~ vs X~ is lost at eps/step per
    iteration (the solve then diverges).
  * U^T V = I is assumed by Step 3 but only inherited through X~ = U X^,
    P~ = U P^ (Section 3.2); rounding errors there grow with the size of
    the coefficients.  Safeguard: when max|U^T V - I| > 1e-12 at Step 3,
    U and V are biorthogonalised again by Alg. 1 (Step 2 applied to the
    current U, V; the search space is unchanged).
  * after a move the projector of eq. hat_pq spans the whole projected
    space (locked pairs + window = all d Ritz pairs), so P^ = 0 exactly and
    P is empty for that iteration (its information is already inside the
    window); computing it anyway only normalises rounding noise.
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------
# operators (matrix-vector products, Section 1 "matrix-free interface")


class DenseOp:
    """K, M (and optionally the SPD B of the generalized LREP, Remark on
    the generalized LREP) stored as dense symmetric matrices.
    Parity: the product is numpy's matmul (a library primitive)."""

    def __init__(self, K, M, B=None):
        self.K = np.asarray(K, dtype=np.float64)
        self.M = np.asarray(M, dtype=np.float64)
        self.B = None if B is None else np.asarray(B, dtype=np.float64)
        self.n = self.K.shape[0]

    def apply(self, which, X):
        if which == "B":
            return X if self.B is None else self.B @ X
        return (self.K if which == "K" else self.M) @ X


class StencilOp:
    """lap_coef * Lap_h + diag(d) on an nx*ny*nz grid, zero ghost values.

    Lap_h x = sum_d (x[+e_d] + x[-e_d] - 2 x) / h^2, index i + nx*(j+ny*k).
    Parity: pinned (separable spectrum = Kronecker sum of the closed-form
    1-D tridiagonal eigenvalues; K phi = 0 for the Gaussian workload).
    """

    def __init__(self, nx, ny, nz, h, lap_coef, dK, dM):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        self.h = h
        self.c = lap_coef / (h * h)
        self.dK = np.asarray(dK, dtype=np.float64)
        self.dM = np.asarray(dM, dtype=np.float64)

    def apply(self, which, X):
        X = np.asarray(X, dtype=np.float64)
        vec = X.ndim == 1
        Xc = X.reshape(self.n, -1)
        c = Xc.shape[1]
        G = Xc.reshape(self.nz, self.ny, self.nx, c)
        L = -6.0 * G
        L[:, :, 1:] += G[:, :, :-1]
        L[:, :, :-1] += G[:, :, 1:]
        L[:, 1:, :] += G[:, :-1, :]
        L[:, :-1, :] += G[:, 1:, :]
        L[1:, :, :] += G[:-1, :, :]
        L[:-1, :, :] += G[1:, :, :]
        d = self.dK if which == "K" else self.dM
        Y = self.c * L.reshape(self.n, c) + d[:, None] * Xc
        return Y[:, 0] if vec else Y


class SpectralOp:
    """lap_coef * Lap_F + diag(d) on a periodic nx*ny*nz grid of a box with
    side lengths L (the Fourier spectral discretisation of the BdG example,
    Section 4, Example "large-scale dense matrix", eq. bdg_KM).

    Lap_F x = ifftn(-|kappa|^2 fftn(x)) over the whole grid, kappa_d =
    2 pi m / L_d for the signed frequencies m of numpy's fftfreq order (the
    Nyquist mode m = -N_d/2 keeps its kappa^2); index i + nx*(j + ny*k).
    Parity: pinned (closed-form Fourier second-derivative matrix, plane
    waves, harmonic-oscillator spectrum, Table 8).
    """

    def __init__(self, nx, ny, nz, L, lap_coef, dK, dM):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        kap = [2.0 * np.pi / float(Ld) * np.fft.fftfreq(Nd, 1.0 / Nd)
               for Nd, Ld in zip((nx, ny, nz), L)]
        k2 = (kap[2][:, None, None] ** 2 + kap[1][None, :, None] ** 2
              + kap[0][None, None, :] ** 2)
        self.mult = -float(lap_coef) * k2  # Fourier multiplier of lap_coef * Lap_F
        self.dK = np.asarray(dK, dtype=np.float64)
        self.dM = np.asarray(dM, dtype=np.float64)

    def apply(self, which, X):
        X = np.asarray(X, dtype=np.float64)
        vec = X.ndim == 1
        Xc = X.reshape(self.n, -1)
        c = Xc.shape[1]
        G = Xc.reshape(self.nz, self.ny, self.nx, c)
        F = np.fft.fftn(G, axes=(0, 1, 2))
        L = np.real(np.fft.ifftn(self.mult[..., None] * F, axes=(0, 1, 2)))
        d = self.dK if which == "K" else self.dM
        Y = L.reshape(self.n, c) + d[:, None] * Xc
        return Y[:, 0] if vec else Y


class CsrOp:
    """K, M given as CSR triples (rowptr, colind, values).
    Parity: pinned (equal to the pinned stencil operator through an
    independent stencil-to-CSR conversion)."""

    def __init__(self, n, csrK, csrM):
        self.n = n
        self.csr = {"K": csrK, "M": csrM}

    def apply(self, which, X):
        rp, ci, va = self.csr[which]
        X = np.asarray(X, dtype=np.float64)
        vec = X.ndim == 1
        Xc = X.reshape(self.n, -1)
        rows = np.repeat(np.arange(self.n), np.diff(rp))
        Y = np.zeros_like(Xc)
        np.add.at(Y, rows, va[:, None] * Xc[ci])
        return Y[:, 0] if vec else Y


# --------------------------------------------------------------------------
# R1: the definition


def lrep_definition(K, M, nev, r=0, FK=None, FM=None):
    """nev smallest positive eigenpairs of H by factorisation + one SVD.

    K = F_K F_K^T, M = F_M F_M^T.  The eigenvalues of H are +-sigma of
    F_K^T F_M (Lemma eigReal: det(lam I - H) = det(lam^2 I - K M) and
    K M is similar to F_K^T F_M F_M^T F_K).  With F_K^T F_M v = sigma w:
    x = F_M v / sqrt(sigma), y = sqrt(sigma) F_M^-T v = F_K w / sqrt(sigma),
    so K x = sigma y, M y = sigma x and x^T y = v^T v = 1.
    The r zero singular values (dim N(K) = r) are dropped.

    Returns (lam ascending, X, Y) with X, Y of shape n x nev.
    Parity: pinned (Example 1 closed form, Table 2/3 values, commuting
    spectra, brute-force eig of H).
    """
    K = np.asarray(K, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    if FK is None:
        kap, Vk = np.linalg.eigh(K)
        FK = Vk * np.sqrt(np.clip(kap, 0.0, None))[None, :]
    if FM is None:
        FM = np.linalg.cholesky(M)
    Wl, sig, Vt = np.linalg.svd(FK.T @ FM)
    order = np.argsort(sig)[r:r + nev]
    sig = sig[order]
    V = Vt.T[:, order]
    Wl = Wl[:, order]
    sq = np.sqrt(sig)
    X = (FM @ V) / sq[None, :]
    Y = (FK @ Wl) / sq[None, :]
    X, Y = fix_sign(X, Y)
    return sig, X, Y


def lrep_definition_gen(K, M, Bm, nev, r=0):
    """Generalized LREP (Remark on the generalized LREP): K x = lam B y,
    M y = lam B x with B symmetric positive definite, x^T B y = 1.

    With B = L L^T: K' = L^-1 K L^-T, M' = L^-1 M L^-T is a standard LREP
    with x' = L^T x, y' = L^T y (K' x' = L^-1 K x = lam L^-1 B y = lam y',
    and x'^T y' = x^T B y), solved by ``lrep_definition``.
    Returns (lam ascending, X, Y) with X, Y of shape n x nev.
    Parity: pinned (B = beta I scales the eigenvalues by 1/beta; the
    eigenvalues of the pencil; K x = lam B y, M y = lam B x, X^T B Y = I).
    """
    L = np.linalg.cholesky(np.asarray(Bm, dtype=np.float64))
    Kp = np.linalg.solve(L, np.linalg.solve(L, np.asarray(K, dtype=np.float64)).T)
    Mp = np.linalg.solve(L, np.linalg.solve(L, np.asarray(M, dtype=np.float64)).T)
    Kp = 0.5 * (Kp + Kp.T)
    Mp = 0.5 * (Mp + Mp.T)
    lam, Xp, Yp = lrep_definition(Kp, Mp, nev, r)
    X = np.linalg.solve(L.T, Xp)
    Y = np.linalg.solve(L.T, Yp)
    X, Y = fix_sign(X, Y)
    return lam, X, Y


def lrep_definition_values(FK, FM, nev, r=0):
    """Eigenvalues only of the definition route (one values-only SVD of
    F_K^T F_M), for orders where the vectors are not needed.
    Parity: pinned against ``lrep_definition`` (same singular values)."""
    sig = np.sort(np.linalg.svd(FK.T @ FM, compute_uv=False))
    return sig[r:r + nev]


def fix_sign(X, Y):
    """Scale pair columns by +-1 so that the largest-|.| entry of x is > 0
    (a sign convention; both sides apply the same one)."""
    X = np.array(X, dtype=np.float64, copy=True)
    Y = np.array(Y, dtype=np.float64, copy=True)
    for i in range(X.shape[1]):
        j = int(np.argmax(np.abs(X[:, i])))
        if X[j, i] < 0:
            X[:, i] *= -1.0
            Y[:, i] *= -1.0
    return X, Y


# --------------------------------------------------------------------------
# Alg. 1 and its classical variant


def mgs_biorth(X, Y, tau=1e-10, ref_norms=None, Bf=None):
    """Alg. 1 (MGS-Biorth) with the discard rule of the Remark after it.

    For l = 1..m: p = x_l, q = y_l; for each kept j < l:
    r_jl = q_j^T p, p -= r_jl p_j, s_jl = p_j^T q, q -= s_jl q_j; then
    eta = p^T q, r_ll = sign(eta) sqrt|eta|, s_ll = sqrt|eta|,
    p_l = p / r_ll, q_l = q / s_ll.  Pairs with |eta| <= tau ||x_l|| ||y_l||
    (or non-finite eta) are dropped; ``ref_norms`` = (||x_l||, ||y_l||)
    arrays replace the input norms when the inputs were projected before.
    ``Bf``: the B-inner product <u, v>_B = u^T B v of the generalized LREP
    (Remark on the generalized LREP), given as v -> B v; norms are then
    B-norms.
    Returns (P, Q, kept indices).
    Parity: pinned (Table 1 losses, P^T Q = I, span checks, LU identity).
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Bf = (lambda v: v) if Bf is None else Bf
    if ref_norms is None:
        ref_norms = (np.sqrt(np.abs(np.sum(X * Bf(X), axis=0))),
                     np.sqrt(np.abs(np.sum(Y * Bf(Y), axis=0))))
    P, Q, kept = [], [], []
    for l in range(X.shape[1]):
        p = X[:, l].copy()
        q = Y[:, l].copy()
        for pj, qj in zip(P, Q):
            r = qj @ Bf(p)
            p -= r * pj
            s = pj @ Bf(q)
            q -= s * qj
        eta = p @ Bf(q)
        bound = tau * ref_norms[0][l] * ref_norms[1][l]
        if not np.isfinite(eta) or abs(eta) <= bound or eta == 0.0:
            continue
        root = np.sqrt(abs(eta))
        P.append(p / (np.sign(eta) * root))
        Q.append(q / root)
        kept.append(l)
    n = X.shape[0]
    if not P:
        return np.zeros((n, 0)), np.zeros((n, 0)), kept
    return np.stack(P, axis=1), np.stack(Q, axis=1), kept


def cgs_biorth(X, Y):
    """Classical (Gauss-Jacobi) Gram-Schmidt biorthogonalisation, Section 3.1.

    Coefficients use the original x, y: r_j = q_j^T x, s_j = p_j^T y.
    Test-only comparator for Table 1 (no discard).
    Parity: pinned (Table 1 losses within 10x).
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    P, Q = [], []
    for l in range(X.shape[1]):
        x = X[:, l]
        y = Y[:, l]
        p = x.copy()
        q = y.copy()
        for pj, qj in zip(P, Q):
            p -= pj * (qj @ x)
            q -= qj * (pj @ y)
        eta = p @ q
        root = np.sqrt(abs(eta))
        P.append(p / (np.sign(eta) * root))
        Q.append(q / root)
    return np.stack(P, axis=1), np.stack(Q, axis=1)


# --------------------------------------------------------------------------
# small LREP (eq. small_eigen)


def small_lrep(Khat, Mhat):
    """All d eigenpairs of the projected LREP [[0, K^], [M^, 0]].

    Two Cholesky factorisations and one SVD (Section 3.3, cost item 2):
    K^ = L1 L1^T, M^ = L2 L2^T, G = L1^T L2 = W S V^T,
    X^ = L2 V S^-1/2, Y^ = L1 W S^-1/2, so that K^ X^ = Y^ S,
    M^ Y^ = X^ S, X^^T Y^ = I.  Returns (lam ascending, X^, Y^) (d x d).
    Raises numpy.linalg.LinAlgError if K^ or M^ is not SPD.
    Parity: pinned (brute-force eig of the 2d x 2d matrix, identities).
    """
    Ks = 0.5 * (Khat + Khat.T)
    Ms = 0.5 * (Mhat + Mhat.T)
    L1 = np.linalg.cholesky(Ks)
    L2 = np.linalg.cholesky(Ms)
    Wl, sig, Vt = np.linalg.svd(L1.T @ L2)
    order = np.argsort(sig)
    sig = sig[order]
    V = Vt.T[:, order]
    Wl = Wl[:, order]
    isq = 1.0 / np.sqrt(sig)
    Xh = (L2 @ V) * isq[None, :]
    Yh = (L1 @ Wl) * isq[None, :]
    return sig, Xh, Yh


# --------------------------------------------------------------------------
# CG and residuals


def cg(apply_fn, B, tol, maxit):
    """Plain CG per column from a zero start (reading of 'tolerance 1e-2,
    at most 20 iterations', text after eq. block_GS).  Columns stop
    independently when ||r|| <= tol ||b||.  Returns (X, iterations run).
    Parity: pinned (reaches ||r|| <= tol ||b|| on an SPD system; exact
    solution within the tolerance)."""
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    R = B.copy()
    P = R.copy()
    rho = np.einsum("ij,ij->j", R, R)
    stop = tol * tol * rho
    active = rho > stop
    it = 0
    while it < maxit and active.any():
        it += 1
        Q = apply_fn(P)
        pq = np.einsum("ij,ij->j", P, Q)
        alpha = np.where(active, rho / np.where(pq == 0, 1.0, pq), 0.0)
        X += P * alpha[None, :]
        R -= Q * alpha[None, :]
        rho_new = np.einsum("ij,ij->j", R, R)
        beta = np.where(active, rho_new / np.where(rho == 0, 1.0, rho), 0.0)
        P = np.where(active[None, :], R + P * beta[None, :], P)
        rho = np.where(active, rho_new, rho)
        active = active & (rho > stop)
    return X, it


def residuals(op, X, Y, lam, KX=None, MY=None, BX=None, BY=None):
    """eq. tol: ||H xi - lam xi|| / ((1 + lam) ||xi||), xi = [y; x]; for the
    generalized LREP H xi - lam diag(B, B) xi.

    KX, MY (BX, BY) may be passed when already formed (K U X^ = (K U) X^).
    Parity: pinned (hand-computed values)."""
    KX = op.apply("K", X) if KX is None else KX
    MY = op.apply("M", Y) if MY is None else MY
    gen = getattr(op, "B", None) is not None
    BX = (op.apply("B", X) if gen else X) if BX is None else BX
    BY = (op.apply("B", Y) if gen else Y) if BY is None else BY
    R1 = KX - BY * lam[None, :]
    R2 = MY - BX * lam[None, :]
    num = np.sqrt(np.sum(R1 * R1, axis=0) + np.sum(R2 * R2, axis=0))
    den = (1.0 + lam) * np.sqrt(np.sum(X * X, axis=0) + np.sum(Y * Y, axis=0))
    return num / den


def nullspace_definition(K, tol):
    """Orthonormal basis of N(K) for symmetric positive semi-definite K, by
    definition: the eigenvectors of K whose eigenvalues are at most
    tol * ||K||_2 (the pre-step of the Remark on the numerical computation
    of the generalized nullspace, which leaves the symmetric eigensolver
    open).  Returns X0 (n x r) and all eigenvalues ascending.
    Parity: pinned (a chosen kernel is recovered, a near-kernel above the
    threshold is not, the zero matrix)."""
    w, V = np.linalg.eigh(np.asarray(K, dtype=np.float64))
    nrm = np.abs(w).max() if w.size else 0.0
    keep = w <= tol * nrm
    return V[:, keep].copy(), w


def setup_nullspace(op, X0, Y0=None, cg_tol=1e-14, cg_maxit=50000):
    """Biorthogonal basis of the generalized nullspace V0.

    Y0 solves M Y0 = X0 (Remark "numerical computation of generalized
    nullspace": CG on the SPD system) unless given; then with
    X0^T Y0 = C^T C (Cholesky), X0 <- X0 C^-1, Y0 <- Y0 C^-1 (eq. V0_basis)
    so that X0^T Y0 = I.  Generalized LREP: M Y0 = B X0 and X0^T B Y0 = I.
    Parity: pinned (Example 2 closed form y0_l = l (n - l + 1) / 2).
    """
    X0 = np.asarray(X0, dtype=np.float64).reshape(op.n, -1)
    gen = getattr(op, "B", None) is not None
    BX0 = op.apply("B", X0) if gen else X0
    if Y0 is None:
        if isinstance(op, DenseOp):
            Y0 = np.linalg.solve(op.M, BX0)
        else:
            Y0, _ = cg(lambda Z: op.apply("M", Z), BX0, cg_tol, cg_maxit)
    Y0 = np.asarray(Y0, dtype=np.float64).reshape(op.n, -1)
    C = np.linalg.cholesky(BX0.T @ Y0).T
    X0 = np.linalg.solve(C.T, X0.T).T
    Y0 = np.linalg.solve(C.T, Y0.T).T
    return X0, Y0


# --------------------------------------------------------------------------
# R2: Alg. 2 with batching and moving


class BospResult(dict):
    __getattr__ = dict.__getitem__


def bosp(op, nev, block, tol, X0=None, Y0=None, start=None, s=3, ngs=1,
         cg_tol=1e-2, cg_maxit=20, maxit=500, discard_tol=1e-10, seed=0,
         max_iters=None, rebiorth_tol=1e-12):
    """Literal Alg. 2 (BOSP) with batching and the moving window.

    ``start``: (U0, V0), n x (w + 2 nb) random blocks for Step 1; drawn
    by ``oracle.philox.normal_block`` (streams 0 and 1) when omitted.
    ``max_iters`` stops early (bounded CPU samples); the result then
    reports only what converged.
    Returns a dict with lam, X, Y (n x nconv), nconv, iters, matvecs,
    history (per-iteration residual lists).
    Parity: pinned against R1 (configs, Examples 1 and 2).
    """
    n = op.n
    nb = min(block, nev)
    moving = nb < nev
    r = 0 if X0 is None else np.asarray(X0).reshape(n, -1).shape[1]
    w = min(s * nb if moving else nev, n - r)
    Kf = lambda Z: op.apply("K", Z)
    Mf = lambda Z: op.apply("M", Z)
    # generalized LREP (Remark on the generalized LREP): every
    # biorthogonality is in the B-inner product u^T B v
    gen = getattr(op, "B", None) is not None
    Bf = (lambda Z: op.apply("B", Z)) if gen else (lambda Z: Z)
    matvecs = 0
    if r:
        X0, Y0 = setup_nullspace(op, X0, Y0)
        Q0, _ = np.linalg.qr(X0)
        Dx, Dy = X0.copy(), Y0.copy()
    else:
        Q0 = None
        Dx, Dy = np.zeros((n, 0)), np.zeros((n, 0))
    # Step 1: random U = [X, P, W], V = [Y, Q, Z]
    d0 = min(w + 2 * nb, n - r)
    if start is None:
        from .philox import normal_block
        U = normal_block(n, d0, seed, 0)
        V = normal_block(n, d0, seed, 1)
    else:
        U = np.array(start[0][:, :d0], dtype=np.float64)
        V = np.array(start[1][:, :d0], dtype=np.float64)
    # Step 2: U = (I - X0 Y0^T) U, V = (I - Y0 X0^T) V, then Alg. 1
    U = U - Dx @ (Dy.T @ Bf(U))
    V = V - Dy @ (Dx.T @ Bf(V))
    U, V, _ = mgs_biorth(U, V, discard_tol, Bf=Bf)
    w_prev = min(w, U.shape[1])
    locked_lam = []
    history = []
    rebiorths = 0
    it = 0
    converged_all = False
    limit = maxit if max_iters is None else min(maxit, max_iters)
    while it < limit:
        it += 1
        d = U.shape[1]
        # safeguard: restore U^T V = I (see module readings)
        if np.abs(U.T @ Bf(V) - np.eye(d)).max() > rebiorth_tol:
            U, V, _ = mgs_biorth(U, V, discard_tol, Bf=Bf)
            d = U.shape[1]
            rebiorths += 1
        # Step 3: H^ (eq. hat_H), small LREP, pullback (eq. eigenVector-pullback)
        KU = Kf(U)
        MV = Mf(V)
        matvecs += 2 * d
        lam, Xh, Yh = small_lrep(U.T @ KU, V.T @ MV)
        for j in range(min(w_prev, d)):
            if Xh[j, j] < 0.0:
                Xh[:, j] = -Xh[:, j]
                Yh[:, j] = -Yh[:, j]
        ell = len(locked_lam)
        wv = min(w, d)
        want = min(wv, nev - ell)
        Xt = U @ Xh[:, :wv]
        Yt = V @ Yh[:, :wv]
        # Step 4: residuals (eq. tol); K X~ = (K U) X^, M Y~ = (M V) Y^
        eps = residuals(op, Xt, Yt, lam[:wv], KU @ Xh[:, :wv], MV @ Yh[:, :wv],
                        Bf(Xt), Bf(Yt))
        history.append(eps.copy())
        c = 0
        while c < wv and eps[c] < tol:
            c += 1
        if c >= want:
            locked_lam.extend(lam[:want].tolist())
            Dx = np.hstack([Dx, Xt[:, :want]])
            Dy = np.hstack([Dy, Yt[:, :want]])
            converged_all = True
            break
        win0 = 0
        if moving and c >= 2 * nb:
            # lock 2 nb pairs, the window moves to Ritz pairs 2nb..
            locked_lam.extend(lam[:2 * nb].tolist())
            Dx = np.hstack([Dx, Xt[:, :2 * nb]])
            Dy = np.hstack([Dy, Yt[:, :2 * nb]])
            win0 = 2 * nb
            wv = min(w, d - win0)
            sl = slice(win0, win0 + wv)
            Xt = U @ Xh[:, sl]
            Yt = V @ Yh[:, sl]
            eps = residuals(op, Xt, Yt, lam[sl], KU @ Xh[:, sl], MV @ Yh[:, sl],
                            Bf(Xt), Bf(Yt))
        end = win0 + wv
        active = [win0 + i for i in range(wv) if not eps[i] < tol][:nb]
        # Step 5: eq. hat_pq, small biorth, P~ = U P^, Q~ = V Q^
        Eb = np.zeros((d, len(active)))
        for col, j in enumerate(active):
            if j < w_prev:
                Eb[j, col] = 1.0
        Pa = Xh[:, active] - Eb
        Qa = Yh[:, active] - Eb
        Ph = Pa - Xh[:, :end] @ (Yh[:, :end].T @ Pa)
        Qh = Qa - Yh[:, :end] @ (Xh[:, :end].T @ Qa)
        pq_ref = (np.linalg.norm(Pa, axis=0), np.linalg.norm(Qa, axis=0))
        if win0 > 0:
            Ph, Qh = Ph[:, :0], Qh[:, :0]   # P^ = 0 after a move
            pq_ref = (pq_ref[0][:0], pq_ref[1][:0])
        Ph, Qh, _ = mgs_biorth(Ph, Qh, discard_tol, pq_ref)  # in R^d: U^T B V = I
        Pt = U @ Ph
        Qt = V @ Qh
        # Step 6: eq. block_GS with CG, then eq. update_W / update_Z
        lam_b = lam[active]
        Xb = U @ Xh[:, active]
        Yb = V @ Yh[:, active]
        KXb = KU @ Xh[:, active]
        MYb = MV @ Yh[:, active]
        Wj = np.zeros_like(Xb)
        BXb, BYb = Bf(Xb), Bf(Yb)
        for _ in range(ngs):
            rhs = Bf(Wj) * lam_b[None, :] + (BXb * lam_b[None, :] - MYb)
            Zj, k1 = cg(Mf, rhs, cg_tol, cg_maxit)
            rhs = Bf(Zj) * lam_b[None, :] + (BYb * lam_b[None, :] - KXb)
            if Q0 is not None:
                rhs = rhs - Q0 @ (Q0.T @ rhs)
            Wj, k2 = cg(Kf, rhs, cg_tol, cg_maxit)
            matvecs += (k1 + k2) * len(active)
        A = np.hstack([Dx, Xt, Pt])
        B = np.hstack([Dy, Yt, Qt])
        Wt = Wj - A @ (B.T @ Bf(Wj))
        Zt = Zj - B @ (A.T @ Bf(Zj))
        wz_ref = (np.sqrt(np.abs(np.sum(Wj * Bf(Wj), axis=0))),
                  np.sqrt(np.abs(np.sum(Zj * Bf(Zj), axis=0))))
        Wt, Zt, _ = mgs_biorth(Wt, Zt, discard_tol, wz_ref, Bf=Bf)
        # Step 7
        U = np.hstack([Xt, Pt, Wt])
        V = np.hstack([Yt, Qt, Zt])
        w_prev = wv
    nconv = len(locked_lam)
    lam_out = np.array(locked_lam)
    Xo, Yo = fix_sign(Dx[:, r:r + nconv], Dy[:, r:r + nconv])
    return BospResult(lam=lam_out, X=Xo, Y=Yo, nconv=nconv, iters=it,
                      matvecs=matvecs, history=history,
                      converged=converged_all, rebiorths=rebiorths)
