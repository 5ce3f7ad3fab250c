"""Pins of the oracle's Fourier spectral operator and of the spectral BdG
workload (Section 4, Example "large-scale dense matrix", eq. bdg, bdg_KM,
Table 8) against facts that do not come from the oracle itself:

* the closed-form Fourier second-derivative matrix of a periodic grid
  (Trefethen, Spectral Methods in MATLAB, ch. 3), on each axis, and the
  Kronecker-sum structure of the 3-D Laplacian;
* plane waves as eigenvectors of Lap_F;
* beta = 0: the GPE ground state is the harmonic-oscillator Gaussian with
  mu = sum(gamma) / 2, and the LREP eigenvalues are the oscillator's
  excitation energies n . gamma;
* beta = 100, n = 16^3: the eigenvalues of Table 8's first column.
"""
import math

import numpy as np
import pytest

from conftest import load_golden
from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth


def _d2_closed_form(N, L):
    """Second-derivative matrix of the periodic band-limited interpolant on
    N equispaced points of a period L (N even): diagonal -pi^2/(3 h^2) - 1/6
    and off-diagonal -(-1)^(j-l) / (2 sin^2((j-l) h / 2)) for h = 2 pi / N,
    scaled by (2 pi / L)^2."""
    h = 2.0 * math.pi / N
    D = np.empty((N, N))
    for a in range(N):
        for b in range(N):
            if a == b:
                D[a, b] = -math.pi ** 2 / (3.0 * h * h) - 1.0 / 6.0
            else:
                D[a, b] = -0.5 * (-1.0) ** (a - b) / math.sin((a - b) * h / 2.0) ** 2
    return D * (2.0 * math.pi / L) ** 2


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32])
def test_spectral_second_derivative_closed_form_each_axis(N):
    L = 5.0
    D = _d2_closed_form(N, L)
    z = np.zeros(N)
    for axis in range(3):
        dims = [1, 1, 1]
        dims[axis] = N
        lengths = [1.0, 1.0, 1.0]
        lengths[axis] = L
        op = R.SpectralOp(*dims, lengths, 1.0, z, z)
        A = op.apply("K", np.eye(N))
        assert np.abs(A - D).max() <= 1e-14 * N * N * np.abs(D).max()


def test_spectral_laplacian_is_kronecker_sum():
    nx, ny, nz, L = 8, 4, 2, (3.0, 5.0, 7.0)
    Dx, Dy, Dz = (_d2_closed_form(N, Ld) for N, Ld in zip((nx, ny, nz), L))
    # index i + nx (j + ny k): x fastest, so the x factor is the last kron
    lap = (np.kron(np.eye(nz), np.kron(np.eye(ny), Dx))
           + np.kron(np.eye(nz), np.kron(Dy, np.eye(nx)))
           + np.kron(Dz, np.kron(np.eye(ny), np.eye(nx))))
    rng = np.random.default_rng(0)
    dK, dM = rng.standard_normal(64), rng.standard_normal(64)
    op = R.SpectralOp(nx, ny, nz, L, -0.5, dK, dM)
    n = nx * ny * nz
    X = rng.standard_normal((n, 5))
    np.testing.assert_allclose(op.apply("K", X), -0.5 * lap @ X + dK[:, None] * X,
                               atol=1e-12)
    np.testing.assert_allclose(op.apply("M", X), -0.5 * lap @ X + dM[:, None] * X,
                               atol=1e-12)


def test_spectral_plane_waves():
    nx, ny, nz, L = 16, 8, 4, (2.0, 3.0, 5.0)
    z, y, x = np.meshgrid(*(np.arange(N) * Ld / N for N, Ld in
                            zip((nz, ny, nx), L[::-1])), indexing="ij")
    op = R.SpectralOp(nx, ny, nz, L, -0.5, np.zeros(nx * ny * nz), np.zeros(nx * ny * nz))
    for m in [(0, 0, 0), (1, 0, 0), (3, 2, 1), (-8, 4, 2), (7, -3, -1)]:
        kap = [2.0 * math.pi * mi / Ld for mi, Ld in zip(m, L)]
        u = np.cos(kap[0] * x + kap[1] * y + kap[2] * z).reshape(-1)
        lam = 0.5 * sum(k * k for k in kap)
        np.testing.assert_allclose(op.apply("K", u), lam * u, atol=1e-11 * max(lam, 1.0))


def test_gpe_ground_state_harmonic_oscillator():
    """beta = 0: phi_s is the normalised oscillator Gaussian, mu = sum(gamma)/2,
    and K = L_GP = H_osc - mu (= M) has the spectrum of the oscillator's
    excitation energies n_x gamma_x + n_y gamma_y (here 0, 1, 2, 2, 3, 3, 4,
    4, 4) with the null vector phi_s."""
    dims, L, gam = (32, 32, 1), (12.0, 12.0, 1.0), (1.0, 2.0, 1.0)
    phi, mu, V, res = synth.gpe_ground_state(dims, L, 0.0, gam)
    assert abs(mu - 1.5) < 1e-12 and res < 1e-12
    h = 12.0 / 32
    x = -6.0 + np.arange(32) * h
    g = np.exp(-0.5 * (gam[1] * x[:, None] ** 2 + gam[0] * x[None, :] ** 2)).reshape(-1)
    g /= math.sqrt(h * h * float(g @ g))
    # the periodic box cuts the Gaussian at |x| = 6, where it is e^-18
    assert np.abs(phi - g).max() < 5e-8
    dK = V - mu
    op = R.SpectralOp(*dims, L, -0.5, dK, dK)
    K = op.apply("K", np.eye(phi.size))
    K = 0.5 * (K + K.T)
    assert np.abs(K @ phi).max() < 1e-11 * np.abs(phi).max()
    w = np.linalg.eigvalsh(K)
    np.testing.assert_allclose(w[:9], [0, 1, 2, 2, 3, 3, 4, 4, 4], rtol=0, atol=1e-8)


def _bdg16_definition():
    p = synth.bdg_spectral(16)
    op = R.SpectralOp(16, 16, 16, p["lengths"], p["lap_coef"], p["dK"], p["dM"])
    n = p["n"]
    K = op.apply("K", np.eye(n))
    M = op.apply("M", np.eye(n))
    K, M = 0.5 * (K + K.T), 0.5 * (M + M.T)
    return p, K, M


def test_bdg_spectral_table8_first_column():
    """n = 16^3 (h = h0 = 1): the eight smallest positive eigenvalues by the
    definition route agree with Table 8's first column to the paper's own
    solver accuracy (its lambda_1, lambda_2 are the same discrete eigenvalue
    by the x <-> y symmetry and differ by 3.5e-11 in the table)."""
    tab = load_golden("table8_bdg.txt")[:, 1]
    p, K, M = _bdg16_definition()
    assert p["gpe_residual"] < 1e-13
    kap, Vk = np.linalg.eigh(K)
    assert abs(kap[0]) < 1e-12 and kap[1] > 0.1  # K = L_GP: one null vector phi_s
    assert abs(abs(Vk[:, 0] @ p["phi"]) - 1.0) < 1e-12
    FK = Vk[:, 1:] * np.sqrt(kap[1:])[None, :]
    FM = np.linalg.cholesky(M)
    lam = R.lrep_definition_values(FK, FM, 8)
    np.testing.assert_allclose(lam, tab, rtol=0, atol=2e-10)
    # the x <-> y symmetry makes lambda_1 = lambda_2 exactly
    assert abs(lam[1] - lam[0]) < 1e-12


def test_bosp_on_spectral_operator_vs_definition():
    """The literal Alg. 2 of the oracle on the spectral operator (8^3 grid of
    (-4, 4)^3, beta = 10, deflated by phi_s) agrees with the definition
    route."""
    p = synth.bdg_spectral(8, 8, 8, box=(8.0, 8.0, 8.0), beta=10.0)
    op = R.SpectralOp(8, 8, 8, p["lengths"], -0.5, p["dK"], p["dM"])
    K = op.apply("K", np.eye(512))
    M = op.apply("M", np.eye(512))
    K, M = 0.5 * (K + K.T), 0.5 * (M + M.T)
    kap, Vk = np.linalg.eigh(K)
    FK = Vk[:, 1:] * np.sqrt(kap[1:])[None, :]
    ref = R.lrep_definition_values(FK, np.linalg.cholesky(M), 6)
    out = R.bosp(op, 6, 6, 1e-10, X0=p["phi"][:, None])
    np.testing.assert_allclose(out["lam"], ref, rtol=1e-10)
    assert R.residuals(op, out["X"], out["Y"], out["lam"]).max() < 1e-10


def test_bdg_spectral_input_conventions():
    """The workload generator follows the example's definitions: periodic
    grid x_j = -8 + j h on (-8, 8), h^3 sum phi_s^2 = 1, phi_s peaked at the
    grid point x = 0 (the spectral discretisation is not sign-preserving:
    at h = 1 its tails dip to -1e-4 of the peak), symmetric under x <-> y
    (gamma_x = gamma_y) and under each reflection x -> -x, K phi_s = 0
    through d_K."""
    p = synth.bdg_spectral(16)
    N, h = 16, 1.0
    phi = p["phi_s"].reshape(N, N, N)  # (z, y, x)
    assert abs(h ** 3 * float(np.sum(phi * phi)) - 1.0) < 1e-13
    assert phi[8, 8, 8] == phi.max() and phi.min() > -1e-3 * phi.max()
    np.testing.assert_allclose(phi, np.transpose(phi, (0, 2, 1)), atol=1e-13)
    # x_j = -8 + j: the reflection x -> -x maps index j to (16 - j) mod 16
    ref = np.roll(phi[:, :, ::-1], 1, axis=2)
    np.testing.assert_allclose(phi, ref, atol=1e-13)
    op = R.SpectralOp(N, N, N, p["lengths"], -0.5, p["dK"], p["dM"])
    assert np.abs(op.apply("K", p["phi"])).max() < 1e-12
    # V at the grid corner x = y = z = -8: (64 + 64 + 4 * 64) / 2
    assert abs(p["V"][0] - 192.0) < 1e-12
