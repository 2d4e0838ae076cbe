"""Variable coefficient u_tt = div(a grad u) + f with the mean-coefficient
preconditioner (Section 3, eq. (var coeff wave), eq. (mean-coefftsmat), Example 2):
operator, right-hand side and solves through the C ABI against the oracle."""
import numpy as np
import pytest

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


def faces_flat(faces):
    return np.concatenate([f.ravel() for f in faces])


AF = {1: lambda x: 1.0 + 0.5 * np.sin(3 * x) ** 2,
      2: lambda x, y: (30.0 + np.sin(x) ** 2) * (30.0 + np.sin(y) ** 2),
      3: lambda x, y, z: 2.0 + x * y + np.cos(z)}


@pytest.mark.parametrize("d,N,nt,nrhs", [(1, 63, 64, 2), (2, 63, 64, 1), (2, 127, 128, 1), (3, 63, 64, 1)])
def test_variable_operator_and_rhs(d, N, nt, nrhs):
    tau = 1.0 / nt
    faces = W.face_coefficients(AF[d], d, N)
    abar = W.grid_mean(AF[d], d, N)
    m = N ** d
    x = W.random_field((nrhs, nt, m), seed=1200 + d)
    f = W.random_field((nrhs, nt, m), seed=1201)
    p0 = W.random_field((nrhs, m), seed=1202)
    p1 = W.random_field((nrhs, m), seed=1203)
    with aao.Solver(d, N, nt, tau, 1e-6, c2=abar, nrhs_max=nrhs, variable_coefficient=True) as s:
        s.set_coefficient(cu(faces_flat(faces)))
        xt = cu(x)
        yt = torch.empty_like(xt)
        s.apply_op(xt, yt)
        bt = torch.empty_like(xt)
        s.build_rhs(cu(f), cu(p0), cu(p1), bt)
        torch.cuda.synchronize()
        y = yt.cpu().numpy()
        bg = bt.cpu().numpy()
    for r in range(nrhs):
        ref = OS.apply_YT_var(x[r], faces, d, N, tau)
        assert np.abs(y[r] - ref).max() <= 1e-13 * np.abs(ref).max()
        prob = W.WaveProblem(d, N, nt, 1.0, 1.0, 1e-6, p0[r], p1[r], f[r])
        rb = OS.rhs_b_var(prob, faces)
        assert np.abs(bg[r] - rb).max() <= 1e-13 * np.abs(rb).max()


def test_constant_face_coefficient_equals_constant_operator():
    d, N, nt, c2 = 2, 63, 64, 2.25
    tau = 1.0 / nt
    faces = W.face_coefficients(lambda x, y: np.full_like(x, c2), d, N)
    x = cu(W.random_field((nt, N * N), seed=1300))
    with aao.Solver(d, N, nt, tau, 1e-2, c2=c2, variable_coefficient=True) as s, \
            aao.Solver(d, N, nt, tau, 1e-2, c2=c2) as s0:
        y0 = torch.empty_like(x)
        s0.apply_op(x, y0)
        s.set_coefficient(cu(faces_flat(faces)))
        y1 = torch.empty_like(x)
        s.apply_op(x, y1)
        torch.cuda.synchronize()
        assert (y1 - y0).abs().max().item() <= 1e-13 * y0.abs().max().item()


@pytest.mark.parametrize("N,nt,prec", [(63, 64, 0), (127, 64, 0), (63, 128, 0), (63, 128, 1)])
def test_example2_solve(N, nt, prec):
    """Example 2 through the GPU: same MINRES iteration count as the oracle at tol 1e-6
    (Table 3: 8-10), and a true relative residual 1e-8 solve that matches the oracle."""
    p = W.example2(N, nt, alpha=1e-6)
    faces = W.face_coefficients(p.meta["a"], 2, N)
    abar = W.grid_mean(p.meta["a"], 2, N)
    b = OS.rhs_b_var(p, faces)
    pc = OF.ABACPreconditioner(2, N, nt, p.tau, 1e-6, c2=abar)
    A = lambda v: OS.apply_YT_var(v, faces, 2, N, p.tau)
    xo6, io6 = OM.minres(A, pc.apply, b, rtol=1e-6, maxit=60)
    xo, io = OM.minres(A, pc.apply, b, rtol=1e-8, maxit=60)
    with aao.Solver(2, N, nt, p.tau, 1e-6, c2=abar, precision=prec, variable_coefficient=True) as s:
        s.set_coefficient(cu(faces_flat(faces)))
        bt = torch.empty((nt, N * N), dtype=torch.float64, device="cuda")
        s.build_rhs(cu(p.f), cu(p.psi0), cu(p.psi1), bt)
        torch.cuda.synchronize()
        assert np.abs(bt.cpu().numpy() - b).max() <= 1e-13 * np.abs(b).max()
        xt = torch.empty_like(bt)
        if prec == 0:
            st, info = s.solve(bt, xt, rtol=1e-6, maxit=60)
            assert st == aao.AAO_OK and abs(info[0]["iters"] - io6["iters"]) <= 1
            assert 8 <= info[0]["iters"] <= 10
        st, info = s.solve(bt, xt, rtol=1e-8, maxit=200)
        torch.cuda.synchronize()
        xg = xt.cpu().numpy()
    assert st == aao.AAO_OK, info
    rel = np.linalg.norm(b - A(xg)) / np.linalg.norm(b)
    assert rel <= 1.001e-8
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-6
    if prec == 0:
        assert abs(info[0]["iters"] - io["iters"]) <= 1
