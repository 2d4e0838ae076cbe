"""MINRES scalar steps fused into the kernels that produce their partial sums (the last
block of each right-hand side runs the step) give the same bits as the separate
one-warp launches, in the host-driven loop and in the graph-captured loop, in every
precision and for the variable-coefficient (physical-basis) solve; and they take three
launches out of every iteration (the loop condition of a graph trip too)."""
import numpy as np
import pytest

import workloads as W

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


def _solve(monkeypatch, fused, graph, d, N, nt, nrhs, prec, alpha, rtol, maxit, var=None):
    monkeypatch.setenv("AAO_FUSED_SCALARS", "1" if fused else "0")
    m = N ** d
    kw = dict(precision=prec, nrhs_max=nrhs, graph=graph)
    if var is not None:
        kw.update(variable_coefficient=True, c2=var[1])
    with aao.Solver(d, N, nt, 1.0 / nt, alpha, **kw) as s:
        if var is not None:
            s.set_coefficient(cu(var[0]))
        x = W.random_field((nrhs, nt, m), seed=2100 + N + nrhs)
        xt = cu(x)
        b = torch.empty_like(xt)
        s.apply_op(xt, b)
        torch.cuda.synchronize()
        out = []
        for _ in range(2):  # the second solve reuses the captured graph
            y = torch.empty_like(xt)
            l0 = s.launches
            st, info = s.solve(b, y, rtol=rtol, maxit=maxit)
            torch.cuda.synchronize()
            out.append((st, [i["iters"] for i in info], [i["status"] for i in info],
                        [i["relres_true"] for i in info], y.cpu().numpy(), s.launches - l0))
    return out


CASES = [
    (1, 63, 64, 1, aao.AAO_PREC_FP64, 1e-6),
    (2, 63, 64, 3, aao.AAO_PREC_FP64, 1e-6),
    (3, 63, 64, 2, aao.AAO_PREC_FP64, 1e-2),
    (2, 127, 128, 1, aao.AAO_PREC_FP32_IR, 1e-3),
    (2, 63, 128, 2, aao.AAO_PREC_F32X2, 1e-6),
]


@pytest.mark.parametrize("d,N,nt,nrhs,prec,alpha", CASES)
@pytest.mark.parametrize("graph", [False, True])
def test_fused_scalars_same_bits(monkeypatch, d, N, nt, nrhs, prec, alpha, graph):
    ref = _solve(monkeypatch, False, graph, d, N, nt, nrhs, prec, alpha, 1e-10, 100)
    fus = _solve(monkeypatch, True, graph, d, N, nt, nrhs, prec, alpha, 1e-10, 100)
    for (st0, it0, ss0, rr0, y0, l0), (st1, it1, ss1, rr1, y1, l1) in zip(ref, fus):
        assert st0 == st1 == aao.AAO_OK
        assert it0 == it1 and ss0 == ss1 and rr0 == rr1
        assert np.array_equal(y0, y1)
        assert l1 < l0
    assert aao.aao_wait_timeouts() == 0


@pytest.mark.parametrize("graph", [False, True])
def test_fused_scalars_variable_coefficient(monkeypatch, graph):
    """Physical-basis solve: the operator's residual mode carries the stop test."""
    N, nt = 63, 64
    p = W.example2(N, nt)
    faces = W.face_coefficients(p.meta["a"], 2, N)
    flat = np.concatenate([f.ravel() for f in faces])
    abar = W.grid_mean(p.meta["a"], 2, N)
    ref = _solve(monkeypatch, False, graph, 2, N, nt, 1, aao.AAO_PREC_FP64, 1e-6, 1e-9, 60, (flat, abar))
    fus = _solve(monkeypatch, True, graph, 2, N, nt, 1, aao.AAO_PREC_FP64, 1e-6, 1e-9, 60, (flat, abar))
    for (st0, it0, ss0, rr0, y0, l0), (st1, it1, ss1, rr1, y1, l1) in zip(ref, fus):
        assert st0 == st1 == aao.AAO_OK
        assert it0 == it1 and rr0 == rr1
        assert np.array_equal(y0, y1)
        assert l1 < l0


@pytest.mark.parametrize("graph", [False, True])
def test_fused_scalars_launches_per_iteration(monkeypatch, graph):
    """Exactly ten iterations (rtol below reach, maxit 10): the fused loop saves three
    launches per iteration (the scalar steps 1, 2, 3) and, in the graph, the loop
    condition of each of its five trips: 30 fewer launches host-driven, 35 in the graph.
    That leaves five launches per iteration in the DST basis."""
    ref = _solve(monkeypatch, False, graph, 2, 63, 64, 1, aao.AAO_PREC_FP64, 1e-2, 1e-300, 10)
    fus = _solve(monkeypatch, True, graph, 2, 63, 64, 1, aao.AAO_PREC_FP64, 1e-2, 1e-300, 10)
    for (st0, it0, ss0, rr0, y0, l0), (st1, it1, ss1, rr1, y1, l1) in zip(ref, fus):
        assert it0 == it1 == [10]
        assert st0 == st1 == aao.AAO_ENOTCONV
        assert np.array_equal(y0, y1)
        assert l0 - l1 == (35 if graph else 30)
