"""Serving: requests of mixed sizes, wave speeds, alpha and tolerances admitted onto
the GPU concurrently under an HBM budget; each result is bit-for-bit the result of
the same solve run alone; budget eviction, an oversize request, bounded waits."""
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


def _solo(p, rtol):
    with aao.Solver(p.d, p.N, p.nt, p.tau, p.alpha, c2=p.c2, graph=True) as s:
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
        with aao.Solver(p.d, p.N, p.nt, p.tau, p.alpha, c2=p.c2, precision=prec, graph=True) as s:
            b = torch.empty((p.nt, p.m), dtype=torch.float64, device="cuda")
            s.build_rhs(f, p0, p1, b)
            xs = torch.empty_like(b)
            st, info = s.solve(b, xs, rtol=r["tol"], maxit=100)
            torch.cuda.synchronize()
        assert st == aao.AAO_OK
        assert res["iters"] == info[0]["iters"]
        assert np.array_equal(x.cpu().numpy(), xs.cpu().numpy()), prec
        assert res["relres_true"] <= r["tol"]
