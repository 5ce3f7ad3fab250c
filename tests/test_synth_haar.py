"""The Householder-form Haar generator behind the n = 32768 mixed-precision
workload (synth.haar_reflectors / loguniform_reflected).

The stored eigenvalues of that workload come from the oracle's definition
route applied to the factors F_K = Q1 diag(sqrt k), F_M = Q2 diag(sqrt m)
formed on the host, while the GPU solves K = F_K F_K^T, M = F_M F_M^T formed
on the device from the same reflectors.  These CPU tests pin what that
relies on: Q is orthogonal and equal to the explicit product of its
reflectors, Q is Haar-distributed (trace moments of the orthogonal group),
and the definition route from the factors equals the route from the formed
matrices.
"""
import math

import numpy as np
import pytest

from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth


def test_reflectors_orthogonal_and_equal_to_explicit_product():
    n = 257
    V, tau, sgn = synth.haar_reflectors(n, np.random.default_rng(5))
    # unit diagonal, zeros above it (LAPACK's storage of the reflectors)
    assert np.all(np.diag(V) == 1.0)
    assert np.all(np.triu(V, 1) == 0.0)
    Q = synth.orthogonal_from_reflectors(V.copy(order="F"), tau, sgn)
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-14
    P = np.eye(n)
    for j in range(n):
        v = V[:, j]
        P = P - tau[j] * np.outer(P @ v, v)
    P *= sgn[None, :]
    assert np.abs(P - Q).max() < 1e-14


def test_reflector_maps_its_draw_to_beta_e1():
    """Each reflector sends its own Gaussian draw x_j to beta_j e_1 with
    sign(beta_j) = sgn[j] and |beta_j| = ||x_j|| (the R diagonal of the
    implied QR)."""
    n = 40
    rng = np.random.default_rng(11)
    V, tau, sgn = synth.haar_reflectors(n, rng)
    draws = np.random.default_rng(11)
    for j in range(n):
        x = draws.standard_normal(n - j)
        v = V[j:, j]
        hx = x - tau[j] * v * (v @ x)
        assert abs(abs(hx[0]) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
        if n - j > 1:
            assert np.abs(hx[1:]).max() < 1e-12 * np.linalg.norm(x)
        assert math.copysign(1.0, hx[0]) == sgn[j]


def test_haar_trace_moments():
    """For Haar-distributed O(n), n >= 4: E tr Q = 0, E (tr Q)^2 = 1,
    E (tr Q)^4 = 3 (Diaconis-Shahshahani); E Q_ij^2 = 1/n.  4000 draws at
    n = 6 put each mean within ~5 standard errors.  Dropping Mezzadri's sign
    fix (sgn = 1) moves E tr Q far from 0 and fails the first check."""
    n, trials = 6, 4000
    rng = np.random.default_rng(2024)
    tr = np.empty(trials)
    tr_nofix = np.empty(trials)
    q11 = np.empty(trials)
    for t in range(trials):
        V, tau, sgn = synth.haar_reflectors(n, rng)
        Q = synth.orthogonal_from_reflectors(V.copy(order="F"), tau, sgn)
        Qn = Q * sgn[None, :]  # undo the sign fix
        tr[t] = np.trace(Q)
        tr_nofix[t] = np.trace(Qn)
        q11[t] = Q[0, 0] ** 2
    se = 1.0 / math.sqrt(trials)
    assert abs(tr.mean()) < 5 * se
    assert abs((tr ** 2).mean() - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs((tr ** 4).mean() - 3.0) < 5 * math.sqrt(96.0) * se
    assert abs(q11.mean() - 1.0 / n) < 5 * math.sqrt(2.0 / (n * (n + 2))) * se
    assert abs(tr_nofix.mean()) > 20 * se


def test_loguniform_spectra_and_factor_route():
    """Spectra lie in [1e-2, 1e2] with log-uniform moments; the definition
    route from the factors equals the one from the formed K, M (eigh and
    Cholesky of the products) to rounding."""
    n = 300
    g = synth.loguniform_reflected(n, seed=3)
    for spec in (g["k"], g["m"]):
        assert spec.min() >= 1e-2 and spec.max() <= 1e2
        u = (np.log(spec) - math.log(1e-2)) / math.log(1e4)
        assert abs(u.mean() - 0.5) < 5 * math.sqrt(1.0 / 12.0 / n)
    FK = synth.reflected_factor_host(g["V1"].copy(order="F"), g["tau1"], g["sgn1"], g["k"])
    FM = synth.reflected_factor_host(g["V2"].copy(order="F"), g["tau2"], g["sgn2"], g["m"])
    lam_f = R.lrep_definition_values(FK, FM, 20)
    K = FK @ FK.T
    M = FM @ FM.T
    lam_m, _, _ = R.lrep_definition(0.5 * (K + K.T), 0.5 * (M + M.T), 20)
    np.testing.assert_allclose(lam_f, lam_m, rtol=1e-11)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_reflectors_tiny_orders(n):
    V, tau, sgn = synth.haar_reflectors(n, np.random.default_rng(n))
    Q = synth.orthogonal_from_reflectors(V.copy(order="F"), tau, sgn)
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-15
    assert tau[-1] == 0.0
