"""Double-float mode (AAO_PREC_F32X2): P_alpha^{-1} and the DSTs of the solve in pairs
of FP32 numbers on the FP32 pipes, operator and recurrences FP64.  Parity of the DST,
the time pipeline and
P_alpha^{-1} against the FP64 oracle within the error the alpha-scaling implies for
~47-bit arithmetic, every kernel variant, and solves that reach the FP64 true
relative residual 1e-8 checked with the oracle operator."""
import os

import numpy as np
import pytest

import gates
import guards
import workloads as W
from oracle import fast as OF
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


@pytest.mark.parametrize("d,N,nt", [(1, 255, 256), (2, 63, 64), (2, 127, 128), (3, 63, 64)])
@pytest.mark.parametrize("alpha", [1e-1, 1e-3, 1e-6])
def test_f32x2_prec_parity(d, N, nt, alpha):
    tau = 1.0 / nt
    x = W.random_field((nt, N ** d), seed=2300 + N + d)
    ref = OF.ABACPreconditioner(d, N, nt, tau, alpha).apply(x)
    with aao.Solver(d, N, nt, tau, alpha, precision=aao.AAO_PREC_F32X2) as s:
        xt = cu(x)
        zt = guards.guarded_empty(xt.shape)
        s.apply_prec(xt, zt)
        torch.cuda.synchronize()
        err = relerr(zt.cpu().numpy(), ref)
        guards.check(zt)
    assert err < gates.dword("prec", d, N, nt, alpha), err
    # far more accurate than FP32: at least 1e4 times below the FP32 gate
    assert err < 1e-4 * gates.fp32("prec", d, N, nt, alpha)


@pytest.mark.parametrize("d,N,nt", [(2, 63, 64), (1, 511, 512), (1, 255, 1024)])
def test_f32x2_time_variants(d, N, nt, monkeypatch):
    alpha = 1e-3
    tau = 1.0 / nt
    m = N ** d
    x = W.random_field((nt, m), seed=2400 + nt)
    ref = OF.time_part_modes(d, N, nt, tau, alpha, x, np.arange(m))
    # 8..11: interleaved layout without the staged table slice; 12, 13 batched loads;
    # 14: 13 built for 5 CTAs per SM; 30 the one-warp small-problem tile
    for v in list(range(15)) + [30]:
        monkeypatch.setenv("AAO_TIME_VARIANT", f"{v},{v},{v}")
        with aao.Solver(d, N, nt, tau, alpha, precision=aao.AAO_PREC_F32X2) as s:
            xt = cu(x)
            yt = torch.empty_like(xt)
            s.apply_time(xt, yt)
            torch.cuda.synchronize()
            assert relerr(yt.cpu().numpy(), ref) < gates.dword("time", d, N, nt, alpha), v


@pytest.mark.parametrize("N,nt", [(63, 64), (127, 128), (255, 256)])
def test_f32x2_solve_reaches_fp64_tolerance(N, nt):
    p = W.config_2d(N=N, nt=nt, alpha=1e-6)
    res = {}
    for prec in (aao.AAO_PREC_FP64, aao.AAO_PREC_F32X2):
        with aao.Solver(2, N, nt, p.tau, p.alpha, precision=prec, graph=True) as s:
            b = torch.empty((nt, p.m), dtype=torch.float64, device="cuda")
            s.build_rhs(cu(p.f), cu(p.psi0), cu(p.psi1), b)
            x = torch.empty_like(b)
            st, info = s.solve(b, x, rtol=1e-8, maxit=100)
            assert st == aao.AAO_OK, info
            res[prec] = (info[0], x.cpu().numpy())
    info, xs = res[aao.AAO_PREC_F32X2]
    bo = OS.rhs_b(p)
    rel = np.linalg.norm(bo - OS.apply_YT(xs, 2, N, p.tau)) / np.linalg.norm(bo)
    assert rel <= 1e-8 * 1.01, rel
    assert info["iters"] <= res[aao.AAO_PREC_FP64][0]["iters"] + 1
    x64 = res[aao.AAO_PREC_FP64][1]
    assert np.linalg.norm(xs - x64) / np.linalg.norm(x64) < 1e-6


def test_f32x2_batched_and_variable_coefficient():
    """Batched right-hand sides give the single results; the variable-coefficient path
    (physical basis, the full double-float P^{-1} every iteration)
    reaches 1e-8."""
    p = W.config_2d(N=63, nt=64, alpha=1e-6)
    f2 = np.stack([p.f, 2.0 * p.f + 1e-3])
    with aao.Solver(2, 63, 64, p.tau, p.alpha, precision=aao.AAO_PREC_F32X2, nrhs_max=2) as s:
        F = cu(f2)
        P0 = cu(np.stack([p.psi0, p.psi0]))
        P1 = cu(np.stack([p.psi1, p.psi1]))
        b = torch.empty_like(F)
        s.build_rhs(F, P0, P1, b)
        x = torch.empty_like(F)
        st, info = s.solve(b, x, rtol=1e-8, maxit=100)
        assert st == aao.AAO_OK
        x1 = torch.empty_like(F[0])
        st1, info1 = s.solve(b[1].contiguous(), x1, rtol=1e-8, maxit=100)
        assert st1 == aao.AAO_OK
        assert np.array_equal(x[1].cpu().numpy(), x1.cpu().numpy())
    q = W.example2(63, 64, alpha=1e-6)
    afun = q.meta["a"]
    faces = W.face_coefficients(afun, 2, 63)
    with aao.Solver(2, 63, 64, q.tau, q.alpha, c2=W.grid_mean(afun, 2, 63), precision=aao.AAO_PREC_F32X2,
                    variable_coefficient=True) as s:
        s.set_coefficient(cu(np.concatenate([fc.ravel() for fc in faces])))
        b = torch.empty((64, q.m), dtype=torch.float64, device="cuda")
        s.build_rhs(cu(q.f), cu(q.psi0), cu(q.psi1), b)
        x = torch.empty_like(b)
        st, info = s.solve(b, x, rtol=1e-8, maxit=200)
        assert st == aao.AAO_OK, info
        xs = x.cpu().numpy()
    bo = OS.rhs_b_var(q, faces)
    rel = np.linalg.norm(bo - OS.apply_YT_var(xs, faces, 2, 63, q.tau)) / np.linalg.norm(bo)
    assert rel <= 1e-8 * 1.01


@pytest.mark.parametrize("d,N", [(1, 511), (2, 63), (2, 255), (3, 63)])
def test_f32x2_dst_parity(d, N, monkeypatch):
    """The double-float DST-I (both stage plans, every axis) against the oracle's explicit
    DST matrices: ~47-bit accuracy, far below FP32 and near FP64."""
    nt = 64
    x = W.random_field((nt, N ** d), seed=2500 + N + d)
    ref = OF.apply_space(x, OF.dst_matrix(N), d, N)
    for dv in range(9):  # 4..7: interleaved padded layout; 8: the one-warp small-problem tile
        monkeypatch.setenv("AAO_DST_VARIANT", str(dv))
        with aao.Solver(d, N, nt, 1.0 / nt, 0.1, precision=aao.AAO_PREC_F32X2) as s:
            xt = cu(x)
            yt = torch.empty_like(xt)
            s.apply_dst(xt, yt)
            torch.cuda.synchronize()
            assert relerr(yt.cpu().numpy(), ref) < gates.dword("dst", d, N, nt), dv


@pytest.mark.parametrize("scale", [1e-25, 1e-3, 1.0, 1e30])
def test_f32x2_conversions_across_scales(scale):
    """The double <-> double-float conversions in the loads and stores take a fast path
    (bit fields, exponents in [-70, 120]) and a fallback (other exponents): scaled
    inputs that land in each give the same relative accuracy, zeros stay zeros, and
    exactly representable inputs survive the round trip."""
    d, N, nt = 2, 63, 64
    x = W.random_field((nt, N ** d), seed=2600) * scale
    x[5] = 0.0                      # a whole time level of zeros
    ref = OF.apply_space(x, OF.dst_matrix(N), d, N)
    with aao.Solver(d, N, nt, 1.0 / nt, 0.1, precision=aao.AAO_PREC_F32X2) as s:
        xt = cu(x)
        yt = torch.empty_like(xt)
        s.apply_dst(xt, yt)
        torch.cuda.synchronize()
        y = yt.cpu().numpy()
        assert relerr(y, ref) < gates.dword("dst", d, N, nt)
        assert np.all(y[5] == 0.0)
        # U is an involution: applying it again returns x to the same accuracy
        s.apply_dst(yt, yt)
        torch.cuda.synchronize()
        assert relerr(yt.cpu().numpy(), x) < 2 * gates.dword("dst", d, N, nt)
