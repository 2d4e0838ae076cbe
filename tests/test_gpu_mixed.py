"""Mixed precision (FP32/complex64 preconditioner, FP64 operator, recurrences and
outer iterative refinement): parity of the FP32 P_alpha^{-1} against the FP64 oracle
within the FP32 error the alpha-scaling implies, and solves that reach the FP64
true relative residual 1e-8."""
import os

import numpy as np
import pytest

import gates
import guards
import workloads as W
from oracle import fast as OF
from oracle import minres as OM
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


def relerr(a, b):
    e = float(np.abs(a - b).max() / np.abs(b).max())
    log = os.environ.get("AAO_PARITY_LOG")
    if log:
        with open(log, "a") as fh:
            fh.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]}\t{e:.3e}\n")
    return e


@pytest.mark.parametrize("d,N,nt", [(1, 255, 256), (2, 63, 64), (2, 255, 256), (3, 63, 64)])
@pytest.mark.parametrize("alpha", [1e-1, 1e-2, 1e-3, 1e-4, 1e-6])
def test_fp32_prec_parity(d, N, nt, alpha):
    tau = 1.0 / nt
    x = W.random_field((nt, N ** d), seed=1000 + N)
    ref = OF.ABACPreconditioner(d, N, nt, tau, alpha).apply(x)
    with aao.Solver(d, N, nt, tau, alpha, precision=aao.AAO_PREC_FP32_IR) as s:
        xt = cu(x)
        zt = guards.guarded_empty(xt.shape)
        s.apply_prec(xt, zt)
        torch.cuda.synchronize()
        err = relerr(zt.cpu().numpy(), ref)
        guards.check(zt)
    assert err < gates.fp32("prec", d, N, nt, alpha), err


@pytest.mark.parametrize("maker,alpha", [
    (lambda a: W.config_1d(alpha=a), 1e-2), (lambda a: W.config_1d(alpha=a), 1e-6),
    (lambda a: W.config_2d(N=63, nt=64, alpha=a), 1e-2), (lambda a: W.config_2d(N=63, nt=64, alpha=a), 1e-4),
    (lambda a: W.config_2d(N=127, nt=128, alpha=a), 1e-6), (lambda a: W.config_2d(N=255, nt=256, alpha=a), 1e-3),
])
def test_fp32_ir_solve_reaches_fp64_tolerance(maker, alpha):
    p = maker(alpha)
    b = OS.rhs_b(p)
    with aao.Solver(p.d, p.N, p.nt, p.tau, alpha, precision=aao.AAO_PREC_FP32_IR) as s:
        bt = cu(b)
        xt = torch.empty_like(bt)
        st, info = s.solve(bt, xt, rtol=1e-8, maxit=200)
        torch.cuda.synchronize()
        xg = xt.cpu().numpy()
    assert st == aao.AAO_OK, info
    rel = np.linalg.norm(b - OS.apply_YT(xg, p.d, p.N, p.tau)) / np.linalg.norm(b)
    assert rel <= 1.001e-8, rel
    assert abs(info[0]["relres_true"] - rel) <= 1e-3 * rel + 1e-15
    pc = OF.ABACPreconditioner(p.d, p.N, p.nt, p.tau, alpha)
    xo, io = OM.minres(lambda v: OS.apply_YT(v, p.d, p.N, p.tau), pc.apply, b, rtol=1e-8)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-6
    if p.exact is not None:
        E = OS.error_E(xg, p.exact_levels(), p.d, p.h)
        Eo = OS.error_E(xo, p.exact_levels(), p.d, p.h)
        assert abs(E - Eo) <= 1e-3 * Eo


def test_fp32_ir_batched():
    d, N, nt, alpha = 2, 63, 64, 1e-3
    tau = 1.0 / nt
    x = W.random_field((3, nt, N * N), seed=1100)
    with aao.Solver(d, N, nt, tau, alpha, precision=aao.AAO_PREC_FP32_IR, nrhs_max=3) as s:
        xt = cu(x)
        b = torch.empty_like(xt)
        s.apply_op(xt, b)
        y = torch.empty_like(xt)
        st, info = s.solve(b, y, rtol=1e-10, maxit=200)
        torch.cuda.synchronize()
        assert st == aao.AAO_OK, info
        assert all(i["relres_true"] <= 1e-10 for i in info)
        assert np.abs(y.cpu().numpy() - x).max() / np.abs(x).max() < 1e-6
