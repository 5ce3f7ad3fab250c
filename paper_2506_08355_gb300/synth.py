"""Seeded synthetic inputs for the linear response eigenvalue problem (LREP).

This module only builds inputs: matrices K, M (or the stencil coefficients),
nullspace bases and random start blocks.  It holds none of the solver's
arithmetic, so both the CUDA path and the CPU oracle may import it.

Workloads (shapes follow the paper's examples, Section 4):

* ``haar_dense``: K = Q1 diag(k) Q1^T, M = Q2 diag(m) Q2^T with Haar-random
  orthogonal Q1, Q2 (QR of a Gaussian matrix with the sign of diag(R) folded
  into Q, Mezzadri's recipe) and spectra k, m drawn uniform or log-uniform.
  Setting some k to zero gives K a known nullspace spanned by the matching
  columns of Q1 (Lemma "generalized nullspace": zero eigenvalues of H).
* ``tridiag_T``: the matrices T(s) of Examples 1 and 2 (1-D finite
  differences; T(0) Dirichlet, T(-1) periodic and singular).
* ``bdg_stencil``: a 7-point finite-difference analogue of the 3-D BdG
  example (Example "large-scale dense matrix"): K = -1/2 Lap_h + d_K,
  M = -1/2 Lap_h + d_M on a cell-centred grid in (-1/2, 1/2)^3 with a
  Dirichlet (zero ghost) boundary.  The condensate phi is a Gaussian of
  widths 1/sqrt(omega0*gamma_d), gamma = (1, 1, 2), normalised to
  h^3 sum phi^2 = 1, and d_K is chosen pointwise as (1/2 Lap_h phi)/phi so
  that K phi = 0 exactly: phi is K's null vector, as the condensate is for
  L_GP in the paper.  d_M = d_K + 2 g phi^2 (the B = g phi^2 coupling).
* ``bdg_spectral``: the BdG example itself in its Fourier spectral form on
  the periodic box (-8, 8)^3 (beta = 100, gamma = (1, 1, 2)), around the
  discrete Gross-Pitaevskii ground state from ``gpe_ground_state`` (a
  nonlinear input solve with its own FFT Laplacian; it is not the
  eigensolver's operator product, which the oracle and the CUDA path each
  implement).
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------
# dense Haar-built problems


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal n x n matrix (QR of N(0,1), signs fixed)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    q *= np.sign(np.diag(r))[None, :]
    return q


def _draw_spectrum(rng, n, lo, hi, law):
    if law == "uniform":
        return rng.uniform(lo, hi, size=n)
    if law == "loguniform":
        return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))
    raise ValueError(law)


def haar_dense(n: int, seed: int, k_range=(0.5, 10.0), m_range=(0.5, 10.0),
               law: str = "uniform", n_zero_k: int = 0, commuting: bool = False):
    """Dense K, M built from chosen spectra and Haar bases.

    Returns a dict with K, M (n x n float64, symmetric), the spectra k, m,
    the bases Q1, Q2 and X0 = Q1[:, :n_zero_k] (the nullspace of K; the
    first ``n_zero_k`` entries of k are set to zero after the draw).
    With ``commuting=True`` Q2 = Q1, so K and M share eigenvectors.
    """
    rng = np.random.default_rng(seed)
    q1 = haar_orthogonal(n, rng)
    q2 = q1 if commuting else haar_orthogonal(n, rng)
    k = _draw_spectrum(rng, n, *k_range, law)
    m = _draw_spectrum(rng, n, *m_range, law)
    k[:n_zero_k] = 0.0
    K = (q1 * k[None, :]) @ q1.T
    M = (q2 * m[None, :]) @ q2.T
    K = 0.5 * (K + K.T)
    M = 0.5 * (M + M.T)
    return {"K": K, "M": M, "k": k, "m": m, "Q1": q1, "Q2": q2,
            "X0": q1[:, :n_zero_k].copy(), "r": n_zero_k}


def haar_dense_device(n: int, seed: int, k_range=(0.5, 10.0), m_range=(0.5, 10.0),
                      law: str = "uniform", n_zero_k: int = 0, device="cuda",
                      gen_dtype="float32"):
    """The same construction as ``haar_dense`` generated on a CUDA device
    with torch (for orders where a host QR takes too long): Gaussian
    matrices from torch's seeded generator, QR with the sign of diag(R)
    folded into Q, spectra from numpy's seeded generator.  With
    gen_dtype float32 the QR and Q diag Q^T run in float32 (seconds at
    n = 32768 instead of minutes) and the result is converted to float64 and
    symmetrised: K, M are then exactly symmetric with eigenvalues within
    ~1e-6 relative of k, m.  Returns torch float64 device tensors K, M, X0
    and numpy k, m."""
    import torch
    gdt = torch.float32 if gen_dtype == "float32" else torch.float64
    g = torch.Generator(device=device).manual_seed(seed)
    rng = np.random.default_rng(seed)
    k = _draw_spectrum(rng, n, *k_range, law)
    m = _draw_spectrum(rng, n, *m_range, law)
    k[:n_zero_k] = 0.0
    out = {}
    for name, spec in (("K", k), ("M", m)):
        G = torch.randn(n, n, dtype=gdt, device=device, generator=g)
        Q, R = torch.linalg.qr(G)
        del G
        Q *= torch.sign(torch.diagonal(R))[None, :]
        del R
        ev = torch.from_numpy(spec).to(device=device, dtype=gdt)
        A = ((Q * ev[None, :]) @ Q.T).to(torch.float64)
        A = 0.5 * (A + A.T)
        out[name] = A
        if name == "K":
            out["X0"] = Q[:, :n_zero_k].to(torch.float64).clone()
        del Q
    out.update(k=k, m=m, r=n_zero_k)
    return out


def haar_reflectors(n: int, rng: np.random.Generator):
    """Householder form of a Haar-random orthogonal n x n matrix, drawn
    directly (Stewart's construction, SIAM J. Numer. Anal. 17, 1980).

    Householder QR of a Gaussian matrix meets, at step j, a column whose
    rows j..n-1 are again N(0, I) and independent of the reflectors before
    it (orthogonal invariance), so drawing that column fresh gives the same
    distribution.  Reflector j maps x_j ~ N(0, I_{n-j}) to beta_j e_1 in
    LAPACK's convention (H_j = I - tau_j v_j v_j^T, v_j[0] = 1,
    beta_j = -sign(x_j[0]) ||x_j||), and Q = H_0 H_1 ... H_{n-1} diag(sign
    beta) is Haar (Mezzadri's sign fix of diag(R)).  Every reflector is a
    well-conditioned function of its own draw, so two machines that form Q
    from the same draws agree to a few units of rounding (a QR of the drawn
    Gaussian matrix would not: its Q moves with the matrix's condition).

    Returns (V, tau, sgn): V n x n Fortran-ordered with v_j in rows j.. of
    column j (unit entry on the diagonal, zeros above), tau and sgn of
    length n."""
    V = np.zeros((n, n), dtype=np.float64, order="F")
    tau = np.zeros(n)
    sgn = np.ones(n)
    for j in range(n):
        x = rng.standard_normal(n - j)
        alpha = float(x[0])
        xnorm = float(np.sqrt(np.dot(x[1:], x[1:]))) if n - j > 1 else 0.0
        if xnorm == 0.0:
            beta = alpha
            V[j, j] = 1.0
        else:
            beta = -math.copysign(math.hypot(alpha, xnorm), alpha)
            tau[j] = (beta - alpha) / beta
            V[j + 1:, j] = x[1:] * (1.0 / (alpha - beta))
            V[j, j] = 1.0
        sgn[j] = 1.0 if beta > 0.0 else -1.0
    return V, tau, sgn


def orthogonal_from_reflectors(V, tau, sgn):
    """Q = H_0 ... H_{n-1} diag(sgn) on the host (LAPACK dorgqr, blocked);
    V is overwritten."""
    from scipy.linalg import lapack
    n = V.shape[0]
    q, _, info = lapack.dorgqr(V, tau, lwork=max(1, 64 * n), overwrite_a=1)
    if info != 0:
        raise RuntimeError("dorgqr info %d" % info)
    q *= sgn[None, :]
    return q


def loguniform_reflected(n: int, seed: int, lo: float = 1e-2, hi: float = 1e2):
    """Inputs of the dense mixed-precision workload: two Haar bases in
    Householder form (``haar_reflectors``) and spectra k, m log-uniform in
    [lo, hi], all from one seeded generator in that order.  K = Q1 diag(k)
    Q1^T and M = Q2 diag(m) Q2^T, i.e. K = F_K F_K^T with
    F_K = Q1 diag(sqrt k) (and F_M alike): the factors the definition route
    takes.  Returns a dict with V1, tau1, sgn1, V2, tau2, sgn2, k, m."""
    rng = np.random.default_rng(seed)
    V1, t1, s1 = haar_reflectors(n, rng)
    V2, t2, s2 = haar_reflectors(n, rng)
    k = _draw_spectrum(rng, n, lo, hi, "loguniform")
    m = _draw_spectrum(rng, n, lo, hi, "loguniform")
    return {"V1": V1, "tau1": t1, "sgn1": s1, "V2": V2, "tau2": t2, "sgn2": s2,
            "k": k, "m": m, "n": n}


def reflected_factor_host(V, tau, sgn, spec):
    """F = Q diag(sqrt(spec)) on the host (V is overwritten)."""
    q = orthogonal_from_reflectors(V, tau, sgn)
    q *= np.sqrt(spec)[None, :]
    return q


def reflected_operator_device(V, tau, sgn, spec, device="cuda"):
    """A = Q diag(spec) Q^T in float64 on a CUDA device with torch (the
    input preparation of the workload, not the solver): Q from the
    reflectors by torch.linalg.householder_product, F = Q diag(sqrt spec),
    A = F F^T symmetrised.  Returns a contiguous float64 device tensor."""
    import torch
    Vd = torch.from_numpy(V).to(device)
    td = torch.from_numpy(np.asarray(tau)).to(device)
    Q = torch.linalg.householder_product(Vd, td)
    del Vd
    scale = torch.from_numpy(np.asarray(sgn) * np.sqrt(spec)).to(device)
    Q *= scale[None, :]
    A = Q @ Q.T
    del Q
    A = 0.5 * (A + A.T)
    return A.contiguous()


def tridiag_T(n: int, s: float) -> np.ndarray:
    """T(s): 2 on the diagonal, -1 off it, s in the two corners (Section 4)."""
    t = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    t[0, n - 1] += s
    t[n - 1, 0] += s
    return t


# --------------------------------------------------------------------------
# 7-point BdG-like stencil


def bdg_stencil(nx: int, ny: int = None, nz: int = None, g: float = 1.0,
                omega0: float = 100.0, gamma=(1.0, 1.0, 2.0),
                shift_c: float = None):
    """Stencil coefficients of the BdG-like workload on an nx*ny*nz grid.

    Grid index i + nx*(j + ny*k) (x fastest), h = 1/nx, points
    x_i = -1/2 + (i + 1/2) h.  Returns dict with dK, dM (n vectors), phi
    (the exact null vector of K, unit 2-norm), h and the grid sizes.

    ``shift_c``: if given, d_M = d_K + shift_c instead of d_K + 2 g phi^2
    (with g = 0 this is the separable special case whose spectrum is known
    from 1-D eigenvalues).
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    h = 1.0 / nx
    dims = (nx, ny, nz)
    coords = [-0.5 + (np.arange(d) + 0.5) * h for d in dims]
    omegas = [omega0 * gm for gm in gamma]
    # 1-D factors: phi = prod_d exp(-omega_d x_d^2 / 2); v_d = 1/2 (r+ + r- - 2)/h^2
    phis, vs = [], []
    for x, om, d in zip(coords, omegas, dims):
        phis.append(np.exp(-0.5 * om * x * x))
        rp = np.exp(-0.5 * om * (2.0 * x * h + h * h))   # phi(x+h)/phi(x)
        rm = np.exp(-0.5 * om * (-2.0 * x * h + h * h))  # phi(x-h)/phi(x)
        rp[-1] = 0.0  # zero ghost beyond the last point
        rm[0] = 0.0   # zero ghost before the first point
        vs.append(0.5 * (rp + rm - 2.0) / (h * h))
    # assemble with x fastest: array shape (nz, ny, nx)
    px, py, pz = phis
    vx, vy, vz = vs
    phi = pz[:, None, None] * py[None, :, None] * px[None, None, :]
    dK = vz[:, None, None] + vy[None, :, None] + vx[None, None, :]
    phi = phi.reshape(-1)
    dK = dK.reshape(-1).copy()
    # normalise h^3 sum phi^2 = 1 for the coupling term
    phi_n = phi / math.sqrt(h ** 3 * float(np.dot(phi, phi)))
    if shift_c is not None:
        dM = dK + shift_c
    else:
        dM = dK + 2.0 * g * phi_n * phi_n
    unit = phi / np.linalg.norm(phi)
    return {"dK": dK, "dM": dM, "phi": unit, "h": h, "nx": nx, "ny": ny,
            "nz": nz, "n": nx * ny * nz, "v1d": vs, "coords": coords,
            "lap_coef": -0.5}


# --------------------------------------------------------------------------
# Fourier spectral BdG (Example "large-scale dense matrix", eq. bdg, bdg_KM)


def _spectral_grid(dims, lengths):
    """Periodic grid x_j = -L/2 + j h, h = L / N per axis (x = 0 on a flat
    axis with N = 1; arrays in (z, y, x) order, x fastest) and the squared
    wave numbers of rfftn."""
    nx, ny, nz = dims
    coords = [(-0.5 * Ld + np.arange(Nd) * (Ld / Nd)) if Nd > 1 else np.zeros(1)
              for Nd, Ld in zip(dims, lengths)]
    kap = [2.0 * math.pi / Ld * np.fft.fftfreq(Nd, 1.0 / Nd) for Nd, Ld in zip(dims, lengths)]
    kx2 = (2.0 * math.pi / lengths[0] * np.fft.rfftfreq(nx, 1.0 / nx)) ** 2
    k2 = (kap[2][:, None, None] ** 2 + kap[1][None, :, None] ** 2 + kx2[None, None, :])
    return coords, k2


def gpe_ground_state(dims, lengths=(16.0, 16.0, 16.0), beta=100.0, gamma=(1.0, 1.0, 2.0),
                     flow_tol=1e-5, newton_tol=1e-13):
    """Discrete ground state of the Gross-Pitaevskii equation (eq. gpe) in
    the Fourier spectral discretisation on the periodic box: the positive
    phi_s with h^3 sum phi_s^2 = 1 and
    [-1/2 Lap_F + V + beta phi_s^2] phi_s = mu_s phi_s,
    V = 1/2 sum_d (gamma_d x_d)^2.  It is an input of the BdG workload
    (the condensate the excitations are computed around), not part of the
    eigensolver.

    Computed by a normalised gradient flow (backward-Euler Fourier step
    with a constant stabilising shift) to flow_tol, then Newton steps on
    (phi, mu) with the normalisation constraint; the Newton system is solved
    with two preconditioned CG solves with L + 2 beta phi^2 (SPD near the
    ground state).  Returns (phi_s, mu_s, V, residual max-norm)."""
    dims = tuple(int(d) for d in dims)
    nx, ny, nz = dims
    coords, k2 = _spectral_grid(dims, lengths)
    hvol = float(np.prod([Ld / Nd for Nd, Ld in zip(dims, lengths) if Nd > 1]))
    shape = (nz, ny, nx)
    z, y, x = coords[2][:, None, None], coords[1][None, :, None], coords[0][None, None, :]
    V = 0.5 * ((gamma[0] * x) ** 2 + (gamma[1] * y) ** 2 + (gamma[2] * z) ** 2)
    V = np.broadcast_to(V, shape).copy()

    def half_lap(u):  # -1/2 Lap_F u
        return np.fft.irfftn(0.5 * k2 * np.fft.rfftn(u), s=shape, axes=(0, 1, 2))

    def normalise(u):
        return u / math.sqrt(hvol * float(np.sum(u * u)))

    phi = normalise(np.exp(-0.5 * (gamma[0] * x * x + gamma[1] * y * y + gamma[2] * z * z))
                    * np.ones(shape))
    tau = 0.5
    for _ in range(20000):
        w = V + beta * phi * phi
        alpha = 0.5 * (float(w.max()) + float(w.min()))
        rhs = (1.0 / tau + alpha - w) * phi
        new = normalise(np.fft.irfftn(np.fft.rfftn(rhs) / (1.0 / tau + alpha + 0.5 * k2),
                                      s=shape, axes=(0, 1, 2)))
        step = float(np.abs(new - phi).max())
        phi = new
        if step < flow_tol:
            break

    def pcg(op, b, tol=1e-14, maxit=5000):
        pre = lambda r: np.fft.irfftn(np.fft.rfftn(r) / (0.5 * k2 + 10.0), s=shape,
                                      axes=(0, 1, 2))
        xk = np.zeros_like(b)
        r = b.copy()
        zr = pre(r)
        p = zr.copy()
        rz = float(np.sum(r * zr))
        nb = math.sqrt(float(np.sum(b * b)))
        for _ in range(maxit):
            q = op(p)
            a = rz / float(np.sum(p * q))
            xk += a * p
            r -= a * q
            if math.sqrt(float(np.sum(r * r))) <= tol * nb:
                break
            zr = pre(r)
            rz2 = float(np.sum(r * zr))
            p = zr + (rz2 / rz) * p
            rz = rz2
        return xk

    res = np.inf
    for _ in range(12):
        Aphi = half_lap(phi) + (V + beta * phi * phi) * phi
        mu = hvol * float(np.sum(phi * Aphi))
        F1 = Aphi - mu * phi
        res = float(np.abs(F1).max())
        if res < newton_tol:
            break
        wM = V + 3.0 * beta * phi * phi - mu
        opM = lambda u: half_lap(u) + wM * u
        a = pcg(opM, F1)
        b = pcg(opM, phi)
        dmu = float(np.sum(phi * a)) / float(np.sum(phi * b))
        phi = normalise(phi - a + dmu * b)
    Aphi = half_lap(phi) + (V + beta * phi * phi) * phi
    mu = hvol * float(np.sum(phi * Aphi))
    res = float(np.abs(Aphi - mu * phi).max())
    return phi.reshape(-1), mu, V.reshape(-1), res


def bdg_spectral(nx: int, ny: int = None, nz: int = None, box=(16.0, 16.0, 16.0),
                 beta: float = 100.0, gamma=(1.0, 1.0, 2.0)):
    """The 3-D BdG workload of the paper's "large-scale dense matrix"
    example in its Fourier spectral form: box (-8, 8)^3, beta = 100,
    gamma = (1, 1, 2), n = nx*ny*nz (Table 8: nx = 16, 32, 64, 128, 256 for
    h = h0 ... h0/16).  K = -1/2 Lap_F + dK and M = -1/2 Lap_F + dM with
    dK = V + beta phi_s^2 - mu_s and dM = dK + 2 beta phi_s^2 (eq. bdg_KM:
    K = L_GP, M = L_GP + 2 beta |phi_s|^2), so K phi_s = 0 up to the ground
    state's residual.  Returns dK, dM, phi (unit 2-norm, the null vector of
    K), phi_s (h^3-normalised), mu, V, lengths and the grid sizes."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    dims = (nx, ny, nz)

    def make():
        phi_s, mu, V, res = gpe_ground_state(dims, box, beta, gamma)
        dK = V + beta * phi_s * phi_s - mu
        return {"dK": dK, "dM": dK + 2.0 * beta * phi_s * phi_s, "phi_s": phi_s,
                "mu": mu, "V": V, "gpe_residual": res}

    n = nx * ny * nz
    if n >= 32768:
        key = "bdg_spectral_%dx%dx%d_b%g_g%g_%g_%g_L%g_%g_%g" % (dims + (beta,) + tuple(gamma)
                                                              + tuple(box))
        out = _cached(key, make)
    else:
        out = make()
    phi = out["phi_s"] / np.linalg.norm(out["phi_s"])
    out.update(phi=phi, lengths=np.asarray(box, dtype=np.float64), nx=nx, ny=ny, nz=nz, n=n,
               lap_coef=-0.5, beta=beta, gamma=tuple(gamma))
    return out


def stencil_to_csr(nx, ny, nz, h, lap_coef, diag):
    """The stencil operator lap_coef*Lap_h + diag(diag) as CSR arrays.

    Returns (rowptr int64, colind int32, values float64); rows are sorted
    by column.  Input construction only (used to feed the CSR form).
    """
    n = nx * ny * nz
    c = lap_coef / (h * h)
    idx = np.arange(n, dtype=np.int64)
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    cols, vals, rows = [], [], []
    rows.append(idx); cols.append(idx); vals.append(diag - 6.0 * c)
    for (cond, off) in ((i > 0, -1), (i < nx - 1, 1), (j > 0, -nx),
                        (j < ny - 1, nx), (k > 0, -nx * ny),
                        (k < nz - 1, nx * ny)):
        r = idx[cond]
        rows.append(r); cols.append(r + off); vals.append(np.full(r.size, c))
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals.astype(np.float64)


def dense_to_csr(A: np.ndarray, drop: float = 0.0):
    """CSR arrays of a dense matrix (entries with |a| <= drop omitted)."""
    n = A.shape[0]
    mask = np.abs(A) > drop
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(mask.sum(axis=1))
    r, c = np.nonzero(mask)
    return rowptr, c.astype(np.int32), A[r, c].astype(np.float64)


# --------------------------------------------------------------------------
# random start blocks and the serving trace


def start_block(n: int, ncols: int, seed: int):
    """Two independent N(0,1) blocks (U0, V0), n x ncols, column-major."""
    rng = np.random.default_rng(seed)
    u = np.asfortranarray(rng.standard_normal((n, ncols)))
    v = np.asfortranarray(rng.standard_normal((n, ncols)))
    return u, v


def serving_trace(num: int = 1000, seed: int = 4, rate_hz: float = 200.0,
                  n_lo: int = 256, n_hi: int = 4096, nevs=(4, 8, 16, 32)):
    """Poisson arrivals with log-uniform n and uniform nev."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=num)
    arrivals = np.cumsum(gaps) - gaps[0]
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=num))).astype(int)
    nev = rng.choice(np.asarray(nevs), size=num)
    return [{"t": float(t), "n": int(nn), "nev": int(e), "seed": 1000 + i}
            for i, (t, nn, e) in enumerate(zip(arrivals, ns, nev))]


# --------------------------------------------------------------------------
# the configurations the solver is measured on


def _cached(name, make):
    """Generated arrays are cached under $LREP_SYNTH_CACHE (default a
    per-user directory in the system temp dir) keyed by name."""
    import os
    import tempfile
    base = os.environ.get("LREP_SYNTH_CACHE",
                          os.path.join(tempfile.gettempdir(), "lrep_synth_cache"))
    path = os.path.join(base, name + ".npz")
    if os.path.exists(path):
        try:
            with np.load(path) as z:
                return {k: (z[k] if z[k].ndim else z[k].item()) for k in z.files}
        except Exception:
            pass
    out = make()
    try:
        os.makedirs(base, exist_ok=True)
        tmp = path + ".%d.tmp.npz" % os.getpid()
        np.savez(tmp, **{k: np.asarray(v) for k, v in out.items()})
        os.replace(tmp, path)
    except OSError:
        pass
    return out


def config(idx: int):
    """Problem description of workload ``idx`` (0..3); see module docstring."""
    if idx == 0:
        p = haar_dense(200, seed=0)
        p.update(nev=4, block=4, tol=1e-10, name="dense-fp64-n200")
        return p
    if idx == 1:
        p = _cached("haar_dense_8192_seed1_null4",
                    lambda: haar_dense(8192, seed=1, n_zero_k=4))
        p.update(nev=64, block=16, tol=1e-10, name="dense-fp64-n8192-null4")
        return p
    if idx == 2:
        p = bdg_stencil(64)
        p.update(nev=32, block=16, tol=1e-10, name="stencil-bdg-64^3", r=1,
                 X0=p["phi"][:, None].copy())
        return p
    if idx == 3:
        p = haar_dense(32768, seed=3, k_range=(1e-2, 1e2), m_range=(1e-2, 1e2),
                       law="loguniform")
        p.update(nev=256, block=32, tol=1e-8, name="dense-mixed-n32768")
        return p
    raise ValueError(idx)
