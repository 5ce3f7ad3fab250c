"""The allocation-free Gram entry point (lrep_op_gram_noalloc).

It serves callers that cannot allocate device memory at call time (HBM
reserved up front by another allocator, or loops that cannot take a
cudaMalloc stall).  Through the C ABI, two calls in a row must give the same
Gram as the pooled entry point lrep_op_gram, within the float64 rounding
bound used for the Gram kernel (two orders of summation of a length-n dot
product differ by at most 2 gamma_n |A|^T |B|).  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def _lib():
    from paper_2506_08355_gb300 import build, lrep
    build.build()
    L = lrep.lib()
    f = L.lrep_op_gram_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                  C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]
    return L


def _gram(fn, A, B, G, stream):
    """G is a (b, ldg) tensor: column j of the a x b Gram is row j, with
    ldg - a padding entries after it."""
    n = A.shape[1]
    return fn(n, A.shape[0], B.shape[0], C.c_void_p(A.data_ptr()), n,
              C.c_void_p(B.data_ptr()), n, C.c_void_p(G.data_ptr()), G.shape[1],
              C.c_void_p(stream))


# (n, a, b, ldg): the first two fit the scratch with every row slab the
# pooled Gram uses; (100000, 256, 256) sits at the limit a * b = 65536, where
# the scratch holds 8 slabs of partials and the Gram is computed with fewer,
# longer slabs than the pooled one; ldg > a leaves padding that must stay
# untouched.
SHAPES = ((70001, 40, 33, 40), (5000, 64, 64, 64), (100000, 256, 256, 256),
          (30011, 24, 50, 31))


@pytest.mark.parametrize("n,a,b,ldg", SHAPES)
def test_gram_noalloc_matches_pooled_gram_twice(n, a, b, ldg):
    import torch
    L = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(99 + n)
    A = torch.tensor(rng.standard_normal((a, n)), device="cuda")
    B = torch.tensor(rng.standard_normal((b, n)), device="cuda")
    An, Bn = A.cpu().numpy().T, B.cpu().numpy().T
    g = n * U / (1 - n * U)
    tol = 2.0 * g * (np.abs(An).T @ np.abs(Bn))
    exact = An.T @ Bn
    G_pool = torch.full((b, ldg), np.nan, dtype=torch.float64, device="cuda")
    assert _gram(L.lrep_op_gram, A, B, G_pool, stream) == 0
    gp = G_pool.cpu().numpy()[:, :a].T
    for call in range(2):  # the shared scratch keeps the previous call's partials
        G_free = torch.full((b, ldg), np.nan, dtype=torch.float64, device="cuda")
        assert _gram(L.lrep_op_gram_noalloc, A, B, G_free, stream) == 0, call
        torch.cuda.synchronize()
        gfull = G_free.cpu().numpy()
        gf = gfull[:, :a].T
        assert np.all(np.abs(gf - gp) <= 2.0 * tol), call
        assert np.all(np.abs(gf - exact) <= tol), call
        assert np.all(np.isnan(gfull[:, a:])), "padding written"


def test_gram_noalloc_rejects_oversize():
    import torch
    L = _lib()
    A = torch.zeros((300, 64), dtype=torch.float64, device="cuda")
    G = torch.zeros((300, 300), dtype=torch.float64, device="cuda")
    st = _gram(L.lrep_op_gram_noalloc, A, A, G, torch.cuda.current_stream().cuda_stream)
    assert st == -1
    assert b"scratch" in L.lrep_last_error(None)
