"""Serving: continuous batching of concurrent solves (lrep_server_*).

Each result must be the same alone (a direct solve) and in the mix: the
small projected problems of concurrent solves share launches, but every
reduction has a fixed order, so the eigenpairs agree to the last bit
(checked to 1e-14).
"""
import numpy as np
import pytest

from oracle import lrep_ref as R
from paper_2506_08355_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(built_lib):
    from paper_2506_08355_gb300 import lrep
    return lrep


def _requests():
    # (n, nev, block, precision, seed); the last has a projected problem of
    # order 48 (grid-wide small LREP), the others below 40 (batched)
    return [(300, 4, 4, 0, 21), (512, 8, 8, 1, 22), (400, 16, 4, 0, 23),
            (640, 4, 4, 1, 24), (350, 8, 8, 0, 25), (700, 12, 4, 0, 26),
            (900, 16, 16, 3, 27)]


def _make(L, n, prec, seed):
    p = synth.haar_dense(n, seed=seed)
    prob = L.Problem.dense(p["K"], p["M"])
    prob.set_options(precision=prec, seed=seed)
    return p, prob


def test_results_identical_alone_and_in_the_mix(L):
    alone = []
    for (n, nev, nb, prec, seed) in _requests():
        p, prob = _make(L, n, prec, seed)
        assert prob.solve(nev, nb, 1e-8) == L.OK
        alone.append((prob.eigvals(), prob.vectors()))
        prob.close()
    srv = L.Server(hbm_budget_bytes=8 << 30, max_slots=4)
    probs, tickets, mats = [], [], []
    for (n, nev, nb, prec, seed) in _requests():
        p, prob = _make(L, n, prec, seed)
        probs.append(prob)
        mats.append(p)
        tickets.append(srv.submit(prob, nev, nb, 1e-8))
    for t in tickets:
        assert srv.wait(t, 120000) == L.OK
    batches, jobs, biggest = srv.stats()
    assert batches > 0 and jobs >= batches
    for prob, (lam0, X0), p, req in zip(probs, alone, mats, _requests()):
        lam, X = prob.eigvals(), prob.vectors()
        np.testing.assert_allclose(lam, lam0, rtol=1e-14, atol=0)
        np.testing.assert_allclose(X, X0, rtol=0, atol=1e-14)
        ref, _, _ = R.lrep_definition(p["K"], p["M"], req[1])
        np.testing.assert_allclose(lam, ref, rtol=1e-10)
    srv.close()
    for prob in probs:
        prob.close()
    # shared launches happened while several solves ran
    assert biggest >= 2


def test_admission_by_hbm_budget_and_host_deadline(L):
    """A budget that fits one request at a time serialises admission (each
    request still solves correctly); a wait with a short host deadline
    returns ERR_TIMEOUT without affecting the request."""
    reqs = [(900, 8, 8, 0, 31), (800, 8, 8, 0, 32), (850, 8, 8, 0, 33)]
    made = [_make(L, n, prec, seed) for (n, nev, nb, prec, seed) in reqs]
    fps = [prob.footprint(nev, nb) for (p, prob), (n, nev, nb, _, _) in zip(made, reqs)]
    assert all(f > 0 for f in fps)
    # room for the largest request, not for two
    srv = L.Server(hbm_budget_bytes=max(fps) + min(fps) // 2, max_slots=3)
    tickets = [srv.submit(prob, nev, nb, 1e-8) for (p, prob), (n, nev, nb, _, _) in zip(made, reqs)]
    first = srv.wait(tickets[-1], 0)   # the last request is still queued
    assert first in (L.OK, -6)
    for t in tickets:
        if t == tickets[-1] and first == L.OK:
            continue  # a finished ticket is reported once
        assert srv.wait(t, 120000) == L.OK
    for (p, prob), (n, nev, nb, _, _) in zip(made, reqs):
        ref, _, _ = R.lrep_definition(p["K"], p["M"], nev)
        np.testing.assert_allclose(prob.eigvals(), ref, rtol=1e-10)
        prob.close()
    srv.close()


def test_request_larger_than_budget_rejected(L):
    p, prob = _make(L, 600, 0, 41)
    srv = L.Server(hbm_budget_bytes=1 << 20, max_slots=1)
    with pytest.raises(L.LrepError):
        srv.submit(prob, 8, 8, 1e-8)
    srv.close()
    prob.close()


def test_small_requests_overtake_one_waiting_for_memory(L):
    """Admission by footprint: a large request that does not fit next to a
    running one waits, and smaller requests behind it that fit start
    meanwhile (no head-of-line blocking).  The mix includes projected
    problems of order >= 40 (nev 16 and 24: grid-wide small LREP) and
    batched ones; every result equals its solo solve to the last bit."""
    reqs = [(1500, 16, 16, 0, 51),   # running first (order 48)
            (2600, 24, 24, 0, 52),   # large: waits for memory
            (400, 4, 4, 0, 53),      # small: fits next to the first
            (500, 8, 8, 1, 54)]      # small
    alone = []
    for (n, nev, nb, prec, seed) in reqs:
        p, prob = _make(L, n, prec, seed)
        assert prob.solve(nev, nb, 1e-8) == L.OK
        alone.append((prob.eigvals(), prob.vectors()))
        prob.close()
    made = [_make(L, n, prec, seed) for (n, nev, nb, prec, seed) in reqs]
    fps = [prob.footprint(nev, nb) for (p, prob), (n, nev, nb, _, _) in zip(made, reqs)]
    # room for the first and the two small ones together, or for the large
    # one alone, never for the first and the large one together
    budget = max(fps[0] + fps[2] + fps[3], fps[1]) + 1
    assert fps[0] + fps[1] > budget
    srv = L.Server(hbm_budget_bytes=budget, max_slots=3)
    import time
    t0 = time.perf_counter()
    tickets = [srv.submit(prob, nev, nb, 1e-8)
               for (p, prob), (n, nev, nb, _, _) in zip(made, reqs)]
    done = {}
    while len(done) < len(tickets):
        for k, t in enumerate(tickets):
            if k in done:
                continue
            st = srv.wait(t, 0)
            if st != -6:
                assert st == L.OK, (k, st)
                done[k] = time.perf_counter() - t0
        time.sleep(0.001)
    # the small requests finished before the large one started and ended
    assert done[2] < done[1] and done[3] < done[1], done
    for (p, prob), (lam0, X0) in zip(made, alone):
        np.testing.assert_allclose(prob.eigvals(), lam0, rtol=1e-14, atol=0)
        np.testing.assert_allclose(prob.vectors(), X0, rtol=0, atol=1e-14)
        prob.close()
    srv.close()
