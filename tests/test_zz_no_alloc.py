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
    n = A.shape[1]
    return fn(n, A.shape[0], B.shape[0], C.c_void_p(A.data_ptr()), n,
              C.c_void_p(B.data_ptr()), n, C.c_void_p(G.data_ptr()), A.shape[0],
              C.c_void_p(stream))


def test_gram_noalloc_matches_pooled_gram_twice():
    import torch
    L = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(99)
    for n, a, b in ((70001, 40, 33), (5000, 64, 64)):
        A = torch.tensor(rng.standard_normal((a, n)), device="cuda")
        B = torch.tensor(rng.standard_normal((b, n)), device="cuda")
        G_pool = torch.zeros((b, a), dtype=torch.float64, device="cuda")
        G_free = torch.full((b, a), np.nan, dtype=torch.float64, device="cuda")
        assert _gram(L.lrep_op_gram, A, B, G_pool, stream) == 0
        assert _gram(L.lrep_op_gram_noalloc, A, B, G_free, stream) == 0
        torch.cuda.synchronize()
        An, Bn = A.cpu().numpy().T, B.cpu().numpy().T
        g = n * U / (1 - n * U)
        tol = 2.0 * g * (np.abs(An).T @ np.abs(Bn))
        gp, gf = G_pool.cpu().numpy().T, G_free.cpu().numpy().T
        assert np.all(np.abs(gf - gp) <= 2.0 * tol)
        assert np.all(np.abs(gf - An.T @ Bn) <= tol)


def test_gram_noalloc_rejects_oversize():
    import torch
    L = _lib()
    A = torch.zeros((300, 64), dtype=torch.float64, device="cuda")
    G = torch.zeros((300, 300), dtype=torch.float64, device="cuda")
    st = _gram(L.lrep_op_gram_noalloc, A, A, G, torch.cuda.current_stream().cuda_stream)
    assert st == -1
    assert b"scratch" in L.lrep_last_error(None)
