"""Graph-captured solves (device-side WHILE loop) give bit-identical results to the
host-driven loop: same kernels in the same order on the same buffers."""
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


@pytest.mark.parametrize("d,N,nt,nrhs,prec,alpha", [
    (1, 63, 64, 1, 0, 1e-6), (2, 63, 64, 3, 0, 1e-6), (2, 127, 128, 1, 1, 1e-3), (3, 63, 64, 2, 0, 1e-2),
    (1, 255, 1024, 1, 1, 1e-3),
])
def test_graph_equals_host_loop(d, N, nt, nrhs, prec, alpha):
    m = N ** d
    tau = 1.0 / nt
    x = W.random_field((nrhs, nt, m), seed=1400 + N)
    out = []
    for graph in (False, True):
        with aao.Solver(d, N, nt, tau, alpha, precision=prec, nrhs_max=nrhs, graph=graph) as s:
            xt = cu(x)
            b = torch.empty_like(xt)
            s.apply_op(xt, b)
            res = []
            for _ in range(2):  # second call reuses the captured graph
                y = torch.empty_like(xt)
                st, info = s.solve(b, y, rtol=1e-10, maxit=100)
                torch.cuda.synchronize()
                res.append((st, [i["iters"] for i in info], y.cpu().numpy()))
            out.append(res)
    (st0, it0, y0), (st0b, it0b, y0b) = out[0]
    for st, it, y in out[1]:
        assert st == st0 == aao.AAO_OK
        assert it == it0
        assert np.array_equal(y, y0)
    assert np.abs(y0 - x).max() / np.abs(x).max() < 1e-7


def test_graph_variable_coefficient_and_maxit():
    p = W.example2(63, 64)
    faces = W.face_coefficients(p.meta["a"], 2, 63)
    flat = np.concatenate([f.ravel() for f in faces])
    abar = W.grid_mean(p.meta["a"], 2, 63)
    b = OS.rhs_b_var(p, faces)
    got = []
    for graph in (False, True):
        with aao.Solver(2, 63, 64, p.tau, 1e-6, c2=abar, variable_coefficient=True, graph=graph) as s:
            s.set_coefficient(cu(flat))
            bt = cu(b)
            y = torch.empty_like(bt)
            st, info = s.solve(bt, y, rtol=1e-9, maxit=100)
            y2 = torch.empty_like(bt)
            st2, info2 = s.solve(bt, y2, rtol=1e-14, maxit=3)   # stops at maxit
            torch.cuda.synchronize()
            got.append((st, info[0]["iters"], y.cpu().numpy(), st2, info2[0]["iters"]))
    assert got[0][0] == got[1][0] == aao.AAO_OK
    assert got[0][1] == got[1][1]
    assert np.array_equal(got[0][2], got[1][2])
    assert got[0][3] == got[1][3] == aao.AAO_ENOTCONV
    assert got[0][4] == got[1][4] == 3


def test_graph_tolerance_and_maxit_per_call():
    """rtol and maxit reach the captured graph through device memory: one graph handle
    alternating tolerances and iteration limits stops exactly where the host-driven
    loop does, call after call."""
    d, N, nt = 2, 63, 128
    x = W.random_field((nt, N * N), seed=1450)
    calls = [(1e-6, 100), (1e-11, 100), (1e-11, 2), (1e-6, 100), (1e-9, 3)]
    out = []
    for graph in (False, True):
        with aao.Solver(d, N, nt, 1.0 / nt, 1e-6, graph=graph) as s:
            xt = cu(x)
            b = torch.empty_like(xt)
            s.apply_op(xt, b)
            res = []
            for rtol, maxit in calls:
                y = torch.empty_like(xt)
                st, info = s.solve(b, y, rtol=rtol, maxit=maxit)
                torch.cuda.synchronize()
                res.append((st, info[0]["iters"], info[0]["relres_true"], y.cpu().numpy()))
            out.append(res)
    for (st0, it0, r0, y0), (st1, it1, r1, y1), (rtol, maxit) in zip(out[0], out[1], calls):
        assert st0 == st1 and it0 == it1 and r0 == r1, (rtol, maxit)
        assert np.array_equal(y0, y1)
        assert it1 <= maxit
        assert (st1 == aao.AAO_OK) == (r1 <= rtol)
    assert out[1][2][0] == aao.AAO_ENOTCONV and out[1][2][1] == 2
    assert out[1][0][1] < out[1][1][1]          # the looser tolerance stops earlier


def test_autotune_keeps_results_and_caches(tmp_path):
    """The autotuner only changes speed: after tuning, P^{-1} and the solve still match
    the oracle; the tune file is written and then read back."""
    from oracle import fast as OF
    d, N, nt, alpha = 2, 127, 128, 1e-2
    tau = 1.0 / nt
    x = W.random_field((nt, N * N), seed=1500)
    ref = OF.ABACPreconditioner(d, N, nt, tau, alpha).apply(x)
    tf = str(tmp_path / "tune.txt")
    for _ in range(2):  # measure + write, then read back
        with aao.Solver(d, N, nt, tau, alpha, graph=True) as s:
            s.autotune(tf)
            xt = cu(x)
            zt = torch.empty_like(xt)
            s.apply_prec(xt, zt)
            torch.cuda.synchronize()
            assert np.abs(zt.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-12
    lines = open(tf).read().strip().splitlines()
    assert len(lines) == 1 and lines[0].split()[:4] == ["2", "127", "128", "0"]


@pytest.mark.parametrize("prec", [aao.AAO_PREC_FP64, aao.AAO_PREC_F32X2, aao.AAO_PREC_FP32_IR])
@pytest.mark.parametrize("graph", [True, False])
def test_host_buffer_solve_equals_device_solve(prec, graph):
    """aao_solve_host pipelines its copies with the right-hand side, the DSTs and the
    solve in chunks of time levels; the result is bit for bit the device-buffer solve of
    the same data (two right-hand sides, pinned and pageable host memory)."""
    p = W.config_2d(N=63, nt=128, alpha=1e-3 if prec == aao.AAO_PREC_FP32_IR else 1e-6)
    f2 = np.stack([p.f, 0.5 * p.f + 1e-3])
    p0 = np.stack([p.psi0, -p.psi0])
    p1 = np.stack([p.psi1, p.psi1 + 0.1])
    with aao.Solver(2, p.N, p.nt, p.tau, p.alpha, precision=prec, nrhs_max=2, graph=graph) as s:
        b = torch.empty((2, p.nt, p.m), dtype=torch.float64, device="cuda")
        s.build_rhs(cu(f2), cu(p0), cu(p1), b)
        x = torch.empty_like(b)
        st, info = s.solve(b, x, rtol=1e-9, maxit=100)
        assert st == aao.AAO_OK
        ref = x.cpu().numpy()
        for pinned in (True, False):
            fh = torch.from_numpy(f2.copy())
            uh = torch.empty((2, p.nt, p.m), dtype=torch.float64)
            if pinned:
                fh, uh = fh.pin_memory(), uh.pin_memory()
            st, info2 = s.solve_host(fh, p0.copy(), p1.copy(), uh, rtol=1e-9, maxit=100)
            assert st == aao.AAO_OK
            assert np.array_equal(uh.numpy(), ref), pinned
            assert [i["iters"] for i in info2] == [i["iters"] for i in info]
