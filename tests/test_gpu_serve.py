"""Serving: requests of mixed sizes, wave speeds, alpha and tolerances admitted onto
the GPU concurrently under an HBM budget; each result is bit-for-bit the result of
the same solve run alone; budget eviction, an oversize request, bounded waits."""
import contextlib
import os
import time

import numpy as np
import pytest

import workloads as W
from oracle import system as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_03574_gb300 as aao  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2306_03574_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    aao.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _requests(k=24, seed=77):
    reqs = W.served_requests(count=k, rate=1e9, seed=seed, max_2d_N=127, max_1d_nt=512, max_2d_nt=128)
    out = []
    for r in reqs:
        p = W.served_problem(r, alpha=1e-6)
        out.append((r, p, cu(p.f), cu(p.psi0), cu(p.psi1), torch.empty((p.nt, p.m), dtype=torch.float64,
                                                                       device="cuda")))
    return out


@contextlib.contextmanager
def _standard_tiles():
    """Served handles run their iterations in grouped launches with the standard tiles,
    also where a handle alone would take the small-problem tiles: the solo reference
    solves keep the standard tiles too (AAO_SMALL_TILES=0, read when the handle is
    created) so that their bits can be compared."""
    old = os.environ.get("AAO_SMALL_TILES")
    os.environ["AAO_SMALL_TILES"] = "0"
    try:
        yield
    finally:
        if old is None:
            del os.environ["AAO_SMALL_TILES"]
        else:
            os.environ["AAO_SMALL_TILES"] = old


def _solo(p, rtol):
    with _standard_tiles(), aao.Solver(p.d, p.N, p.nt, p.tau, p.alpha, c2=p.c2, graph=True) as s:
        b = torch.empty((p.nt, p.m), dtype=torch.float64, device="cuda")
        s.build_rhs(cu(p.f), cu(p.psi0), cu(p.psi1), b)
        x = torch.empty_like(b)
        st, info = s.solve(b, x, rtol=rtol, maxit=100)
        torch.cuda.synchronize()
        return st, info[0], x.cpu().numpy()


def test_mixed_requests_equal_solo_solves():
    reqs = _requests()
    srv = aao.aao_serve_create(8 << 30, 6)
    try:
        tickets = [aao.aao_serve_submit(srv, p.d, p.N, p.nt, p.tau, p.alpha, p.c2, r["tol"], 100, f, p0, p1, x)
                   for (r, p, f, p0, p1, x) in reqs]
        results = []
        for t in tickets:
            st, res = aao.aao_serve_wait(srv, t, 120.0)
            assert st == aao.AAO_OK, (st, res)
            results.append(res)
        stats = aao.aao_serve_stats(srv)
    finally:
        aao.aao_serve_destroy(srv)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["peak_pool_bytes"] <= stats["budget"]
    # the iterations ran as grouped launches: more than one request per round on average,
    # and a round's launch count bounded by the step kernels plus one time launch per
    # (precision, n) bucket, whatever the number of requests in it
    assert stats["round_problems"] > stats["rounds"], stats
    assert stats["grouped_launches"] <= stats["rounds"] * (7 + 10), stats
    for (r, p, f, p0, p1, x), res in zip(reqs, results):
        st, info, xs = _solo(p, r["tol"])
        assert st == aao.AAO_OK
        assert res["iters"] == info["iters"]
        assert np.array_equal(x.cpu().numpy(), xs)
        b = OS.rhs_b(p)
        rel = np.linalg.norm(b - OS.apply_YT(xs, p.d, p.N, p.tau, p.c2)) / np.linalg.norm(b)
        assert rel <= r["tol"] * 1.001
        assert res["t_submit"] <= res["t_start"] <= res["t_done"]


def _submit_wait(srv, p, tol=1e-8):
    f, p0, p1 = cu(p.f), cu(p.psi0), cu(p.psi1)
    x = torch.empty((p.nt, p.m), dtype=torch.float64, device="cuda")
    t = aao.aao_serve_submit(srv, p.d, p.N, p.nt, p.tau, p.alpha, p.c2, tol, 100, f, p0, p1, x)
    return aao.aao_serve_wait(srv, t, 120.0)


def test_budget_eviction_and_oversize():
    """Two shapes of nearly equal footprint under a budget that holds only one: every
    switch of shape evicts the idle handle of the other; a request larger than the
    budget completes with AAO_ENOMEM."""
    pa = W.config_2d(N=127, nt=128, alpha=1e-6)
    pb = W.config_2d(N=63, nt=512, alpha=1e-6)
    sizes = []
    for p in (pa, pb):  # the pool bytes one handle of each shape takes
        srv = aao.aao_serve_create(8 << 30, 1)
        try:
            assert _submit_wait(srv, p)[0] == aao.AAO_OK
            sizes.append(aao.aao_serve_stats(srv)["pool_bytes"])
        finally:
            aao.aao_serve_destroy(srv)
    budget = int(1.5 * max(sizes))
    srv = aao.aao_serve_create(budget, 2)
    try:
        for p in (pa, pb, pa, pb):
            assert _submit_wait(srv, p)[0] == aao.AAO_OK
        stats = aao.aao_serve_stats(srv)
        assert stats["peak_pool_bytes"] <= budget
        assert stats["evictions"] >= 3 and stats["handles_created"] == 4
        # a request that can never fit completes with AAO_ENOMEM
        assert _submit_wait(srv, W.config_2d(N=255, nt=512, alpha=1e-6))[0] == aao.AAO_ENOMEM
        # unknown ticket
        assert aao.aao_serve_poll(srv, 123456789)[0] == aao.AAO_EINVAL
    finally:
        aao.aao_serve_destroy(srv)


def test_bounded_wait_times_out_then_completes():
    p = W.config_2d(N=255, nt=256, alpha=1e-6)
    f, p0, p1 = cu(p.f), cu(p.psi0), cu(p.psi1)
    x = torch.empty((p.nt, p.m), dtype=torch.float64, device="cuda")
    srv = aao.aao_serve_create(8 << 30, 2)
    try:
        t = aao.aao_serve_submit(srv, 2, 255, 256, p.tau, 1e-6, 1.0, 1e-8, 100, f, p0, p1, x)
        st, _ = aao.aao_serve_wait(srv, t, 1e-6)
        assert st == aao.AAO_ETIMEOUT
        st, _ = aao.aao_serve_poll(srv, t)
        assert st in (aao.AAO_EPENDING, aao.AAO_OK)
        if st == aao.AAO_EPENDING:
            st, res = aao.aao_serve_wait(srv, t, 120.0)
            assert st == aao.AAO_OK
    finally:
        aao.aao_serve_destroy(srv)


def test_served_precisions_equal_solo_solves():
    """Requests may ask for the double-float mode: FP64 and double-float requests of the
    same shapes get separate pooled handles, and each result equals the same solve run
    alone in its precision, bit for bit (and meets the FP64 true-residual tolerance)."""
    reqs = _requests(k=8, seed=91)
    srv = aao.aao_serve_create(8 << 30, 4)
    try:
        tickets = []
        for i, (r, p, f, p0, p1, x) in enumerate(reqs):
            prec = aao.AAO_PREC_F32X2 if i % 2 else aao.AAO_PREC_FP64
            tickets.append((prec, aao.aao_serve_submit(srv, p.d, p.N, p.nt, p.tau, p.alpha, p.c2, r["tol"], 100,
                                                       f, p0, p1, x, precision=prec)))
        results = []
        for prec, t in tickets:
            st, res = aao.aao_serve_wait(srv, t, 120.0)
            assert st == aao.AAO_OK, (st, res)
            results.append(res)
        with pytest.raises(aao.AaoError):  # the refinement mode is not served
            r, p, f, p0, p1, x = reqs[0]
            aao.aao_serve_submit(srv, p.d, p.N, p.nt, p.tau, p.alpha, p.c2, 1e-8, 100, f, p0, p1, x,
                                 precision=aao.AAO_PREC_FP32_IR)
    finally:
        aao.aao_serve_destroy(srv)
    for (prec, _), (r, p, f, p0, p1, x), res in zip(tickets, reqs, results):
        with _standard_tiles(), aao.Solver(p.d, p.N, p.nt, p.tau, p.alpha, c2=p.c2, precision=prec,
                                           graph=True) as s:
            b = torch.empty((p.nt, p.m), dtype=torch.float64, device="cuda")
            s.build_rhs(f, p0, p1, b)
            xs = torch.empty_like(b)
            st, info = s.solve(b, xs, rtol=r["tol"], maxit=100)
            torch.cuda.synchronize()
        assert st == aao.AAO_OK
        assert res["iters"] == info[0]["iters"]
        assert np.array_equal(x.cpu().numpy(), xs.cpu().numpy()), prec
        assert res["relres_true"] <= r["tol"]


def test_requests_arriving_during_a_solve_are_admitted_and_finish_first():
    """Continuous admission: small requests submitted while a large solve is on the GPU
    start before it finishes and complete before it (their size class has its own
    stream and rounds), and every result equals its solo solve."""
    big = W.config_2d(N=255, nt=512, alpha=1e-6)
    small = [W.served_problem(dict(d=1, N=N, nt=nt, c2=c2, tol=1e-8, seed=3000 + i), alpha=1e-6)
             for i, (N, nt, c2) in enumerate([(63, 64, 1.0), (127, 128, 2.2), (255, 64, 0.5), (63, 256, 1.7)])]
    srv = aao.aao_serve_create(16 << 30, 8)
    try:
        # warm the pool (handles, kernels) so the timing below is the solves'
        for p in [big] + small:
            assert _submit_wait(srv, p)[0] == aao.AAO_OK
        bufs = []
        xb = torch.empty((big.nt, big.m), dtype=torch.float64, device="cuda")
        fb, b0, b1 = cu(big.f), cu(big.psi0), cu(big.psi1)
        tb = aao.aao_serve_submit(srv, 2, big.N, big.nt, big.tau, 1e-6, 1.0, 1e-8, 100, fb, b0, b1, xb)
        time.sleep(2e-3)
        ts = []
        for p in small:
            f, p0, p1 = cu(p.f), cu(p.psi0), cu(p.psi1)
            x = torch.empty((p.nt, p.m), dtype=torch.float64, device="cuda")
            bufs.append((p, f, p0, p1, x))
            ts.append(aao.aao_serve_submit(srv, 1, p.N, p.nt, p.tau, 1e-6, p.c2, 1e-8, 100, f, p0, p1, x))
        st, rb = aao.aao_serve_wait(srv, tb, 120.0)
        assert st == aao.AAO_OK
        rs = []
        for t in ts:
            st, r = aao.aao_serve_wait(srv, t, 120.0)
            assert st == aao.AAO_OK
            rs.append(r)
    finally:
        aao.aao_serve_destroy(srv)
    for r in rs:
        assert r["t_start"] < rb["t_done"], (r, rb)
        assert r["t_done"] < rb["t_done"], (r, rb)
    for (p, f, p0, p1, x), r in zip(bufs, rs):
        st, info, xs = _solo(p, 1e-8)
        assert st == aao.AAO_OK and info["iters"] == r["iters"]
        assert np.array_equal(x.cpu().numpy(), xs)
