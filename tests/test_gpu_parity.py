"""GPU parity: every step of the hot path through the C ABI against the CPU oracle
on the same seeded inputs (element by element), plus invariants at full size."""
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
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    aao.lib()
    yield


DEV = "cuda"


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def relerr(a, b):
    e = float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))
    log = os.environ.get("AAO_PARITY_LOG")
    if log:
        with open(log, "a") as fh:
            fh.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]}\t{e:.3e}\n")
    return e


SIZES = [  # (d, N, nt, nrhs): several tiles, ragged tails (N odd, m odd), batches
    (1, 63, 64, 1), (1, 127, 128, 3), (1, 511, 1024, 1), (1, 255, 512, 2),
    (2, 63, 64, 1), (2, 127, 128, 1), (2, 63, 256, 2), (2, 255, 64, 1),
    (3, 63, 64, 1), (3, 127, 64, 1),
]


@pytest.mark.parametrize("d,N,nt,nrhs", SIZES)
def test_dst_parity(d, N, nt, nrhs):
    m = N ** d
    x = W.random_field((nrhs, nt, m), seed=100 + d * 7 + N)
    S = OF.dst_matrix(N)
    ref = np.stack([OF.apply_space(x[r], S, d, N) for r in range(nrhs)])
    with aao.Solver(d, N, nt, 1.0 / nt, 0.1, nrhs_max=nrhs) as s:
        xt = cu(x)
        yt = guards.guarded_empty(xt.shape)
        s.apply_dst(xt, yt)
        torch.cuda.synchronize()
        assert relerr(yt.cpu().numpy(), ref) < 1e-13
        # U is an involution: applying it twice in place returns x
        s.apply_dst(yt, yt)
        torch.cuda.synchronize()
        assert relerr(yt.cpu().numpy(), x) < 1e-13
        guards.check(yt)


@pytest.mark.parametrize("d,N,nt,nrhs", SIZES[:8])
@pytest.mark.parametrize("alpha", [1e-1, 1e-3, 1e-6])
def test_time_pipeline_parity(d, N, nt, nrhs, alpha):
    """apply_time == U P^{-1} U (U^2 = I), with P^{-1} from the oracle."""
    m = N ** d
    tau = 1.0 / nt
    x = W.random_field((nrhs, nt, m), seed=200 + N + nt)
    pc = OF.ABACPreconditioner(d, N, nt, tau, alpha)
    S = OF.dst_matrix(N)
    ref = np.stack([OF.apply_space(pc.apply(OF.apply_space(x[r], S, d, N)), S, d, N)
                    for r in range(nrhs)])
    with aao.Solver(d, N, nt, tau, alpha, nrhs_max=nrhs) as s:
        xt = cu(x)
        yt = guards.guarded_empty(xt.shape)
        s.apply_time(xt, yt)
        torch.cuda.synchronize()
        assert relerr(yt.cpu().numpy(), ref) < gates.fp64("time", d, N, nt, alpha)
        guards.check(yt)


@pytest.mark.parametrize("d,N,nt,nrhs", SIZES)
@pytest.mark.parametrize("alpha", [1e-1, 1e-2, 1e-3, 1e-6])
def test_prec_parity(d, N, nt, nrhs, alpha):
    """One P_alpha^{-1} application == the oracle's three-step procedure done twice."""
    m = N ** d
    tau = 1.0 / nt
    x = W.random_field((nrhs, nt, m), seed=300 + N + nt + d)
    pc = OF.ABACPreconditioner(d, N, nt, tau, alpha)
    ref = np.stack([pc.apply(x[r]) for r in range(nrhs)])
    with aao.Solver(d, N, nt, tau, alpha, nrhs_max=nrhs) as s:
        xt = guards.guarded_copy(x)
        zt = guards.guarded_empty(xt.shape)
        s.apply_prec(xt, zt)
        torch.cuda.synchronize()
        z = zt.cpu().numpy()
        assert relerr(z, ref) < gates.fp64("prec", d, N, nt, alpha)
        guards.check(zt)
        # in place gives the same bits
        s.apply_prec(xt, xt)
        torch.cuda.synchronize()
        assert np.array_equal(xt.cpu().numpy(), z)
        guards.check(xt)


@pytest.mark.parametrize("d,N,nt,nrhs,c2", [(1, 63, 64, 1, 1.0), (2, 63, 64, 2, 1.0), (2, 255, 256, 1, 1.0),
                                            (3, 63, 64, 1, 0.49), (2, 127, 64, 1, 3.3)])
def test_operator_and_rhs_parity(d, N, nt, nrhs, c2):
    m = N ** d
    tau = 1.0 / nt
    x = W.random_field((nrhs, nt, m), seed=400 + N)
    ref = np.stack([OS.apply_YT(x[r], d, N, tau, c2) for r in range(nrhs)])
    f = W.random_field((nrhs, nt, m), seed=401)
    p0 = W.random_field((nrhs, m), seed=402)
    p1 = W.random_field((nrhs, m), seed=403)
    with aao.Solver(d, N, nt, tau, 0.1, c2=c2, nrhs_max=nrhs) as s:
        xt = cu(x)
        yt = guards.guarded_empty(xt.shape)
        s.apply_op(xt, yt)
        bt = guards.guarded_empty(xt.shape)
        s.build_rhs(cu(f), cu(p0), cu(p1), bt)
        torch.cuda.synchronize()
        assert relerr(yt.cpu().numpy(), ref) < 1e-14
        guards.check(yt)
        for r in range(nrhs):
            prob = W.WaveProblem(d, N, nt, 1.0, c2, 0.1, p0[r], p1[r], f[r])
            assert relerr(bt.cpu().numpy()[r], OS.rhs_b(prob)) < 1e-14
        guards.check(bt)


def _solve_both(p, rtol=1e-8, maxit=60):
    tau = p.tau
    pc = OF.ABACPreconditioner(p.d, p.N, p.nt, tau, p.alpha, p.c2)
    b = OS.rhs_b(p)
    xo, io = OM.minres(lambda v: OS.apply_YT(v, p.d, p.N, tau, p.c2), pc.apply, b, rtol=rtol, maxit=maxit)
    with aao.Solver(p.d, p.N, p.nt, tau, p.alpha, c2=p.c2) as s:
        bt = torch.empty((p.nt, p.m), dtype=torch.float64, device=DEV)
        s.build_rhs(cu(p.f), cu(p.psi0), cu(p.psi1), bt)
        xt = torch.empty_like(bt)
        st, info = s.solve(bt, xt, rtol=rtol, maxit=maxit)
        torch.cuda.synchronize()
        xg = xt.cpu().numpy()
    return b, xo, io, xg, st, info[0]


@pytest.mark.parametrize("maker,alpha", [
    (lambda a: W.config_1d(alpha=a), 1e-6), (lambda a: W.config_1d(alpha=a), 1e-1),
    (lambda a: W.config_1d(alpha=a), 1e-2), (lambda a: W.config_1d(alpha=a), 1e-3),
    (lambda a: W.config_2d(N=63, nt=64, alpha=a), 1e-6),
    (lambda a: W.config_2d(N=127, nt=128, alpha=a, c2=2.0), 1e-6),
    (lambda a: W.example1(63, 64, alpha=a), 1e-6),
])
def test_minres_parity(maker, alpha):
    """Same iterations as the oracle MINRES (true relative residual 1e-8), the GPU
    solution's residual re-checked with the oracle's operator, solutions agree."""
    p = maker(alpha)
    b, xo, io, xg, st, ig = _solve_both(p)
    assert st == aao.AAO_OK, ig
    assert abs(ig["iters"] - io["iters"]) <= 1, (ig, io["iters"])
    rel = np.linalg.norm(b - OS.apply_YT(xg, p.d, p.N, p.tau, p.c2)) / np.linalg.norm(b)
    assert rel <= 1e-8 * 1.001, rel
    assert abs(ig["relres_true"] - rel) <= 1e-3 * rel + 1e-15
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-6


def test_table1_two_iterations_gpu():
    """Table 1 / Table 2 MINRES-P_alpha column on the GPU: tol 1e-6 -> 2 iterations
    and E_{tau,h} = 1.88e-5 at tau = h = 2^-6 (within 1%)."""
    p = W.example1(63, 64, alpha=1e-6)
    b, xo, io, xg, st, ig = _solve_both(p, rtol=1e-6)
    assert ig["iters"] == 2
    E = OS.error_E(xg, p.exact_levels(), 2, p.h)
    assert abs(E - 1.88e-5) <= 0.01 * 1.88e-5


def test_full_size_2d_prec_and_invariants():
    """2D 255^2 x 256 (16.6M unknowns): P^{-1} == oracle element by element; Q_alpha^2 = I;
    <P^{-1}x, y> = <x, P^{-1}y>; deterministic bits."""
    d, N, nt = 2, 255, 256
    tau = 1.0 / nt
    # P^{-1}: the error model at alpha = 1e-2; at alpha = 1e-6 the specification's 1e-9,
    # since the max over 16.6 M entries sits above the small-case model there (measured
    # 1.4e-10).  The invariants' gates sit within 30x of their measured values
    # (Q^2 = I: 1.2e-13 and 6.0e-11).
    for alpha, tol, tol_inv in ((1e-2, gates.fp64("prec", d, N, nt, 1e-2), 1e-12), (1e-6, 1e-9, 1e-9)):
        x = W.random_field((nt, N * N), seed=500)
        pc = OF.ABACPreconditioner(d, N, nt, tau, alpha)
        ref = pc.apply(x)
        with aao.Solver(d, N, nt, tau, alpha) as s:
            xt = cu(x)
            zt = torch.empty_like(xt)
            s.apply_prec(xt, zt)
            z2 = torch.empty_like(xt)
            s.apply_prec(xt, z2)
            torch.cuda.synchronize()
            z = zt.cpu().numpy()
            assert relerr(z, ref) < tol
            assert torch.equal(zt, z2)
            # Q^2 = I with Q = P^{-1} Y C_alpha (Lemma qalphaorthoglm)
            yc = OF.apply_C_alpha_direct(x, d, N, tau, alpha)[::-1].copy()
            q1 = torch.empty_like(xt)
            s.apply_prec(cu(yc), q1)
            torch.cuda.synchronize()
            yc2 = OF.apply_C_alpha_direct(q1.cpu().numpy(), d, N, tau, alpha)[::-1].copy()
            q2 = torch.empty_like(xt)
            s.apply_prec(cu(yc2), q2)
            torch.cuda.synchronize()
            assert relerr(q2.cpu().numpy(), x) < tol_inv
            y = W.random_field((nt, N * N), seed=501)
            py = torch.empty_like(xt)
            s.apply_prec(cu(y), py)
            torch.cuda.synchronize()
            a1 = float(np.vdot(z, y))
            a2 = float(np.vdot(x, py.cpu().numpy()))
            sym = relerr(np.array([a2]), np.array([a1]))
            assert sym < max(1e-12, 1e-13 / alpha)


def test_full_size_2d_solve():
    """The 2D 255^2 x 256 workload: MINRES to true relative residual 1e-8, the residual
    re-checked with the oracle operator, E_{tau,h} vs the exact solution at the
    discretisation level, iteration count equal to the oracle's."""
    p = W.config_2d()
    b, xo, io, xg, st, ig = _solve_both(p)
    assert st == aao.AAO_OK
    assert abs(ig["iters"] - io["iters"]) <= 1
    rel = np.linalg.norm(b - OS.apply_YT(xg, 2, p.N, p.tau)) / np.linalg.norm(b)
    assert rel <= 1.001e-8
    E = OS.error_E(xg, p.exact_levels(), 2, p.h)
    Eo = OS.error_E(xo, p.exact_levels(), 2, p.h)
    assert abs(E - Eo) <= 1e-3 * Eo


def test_batch_equals_single_and_determinism():
    d, N, nt = 2, 63, 128
    tau = 1.0 / nt
    x = W.random_field((3, nt, N * N), seed=600)
    with aao.Solver(d, N, nt, tau, 1e-6, nrhs_max=3) as s:
        xt = cu(x)
        zb = torch.empty_like(xt)
        s.apply_prec(xt, zb)
        singles = []
        for r in range(3):
            zr = torch.empty_like(xt[r])
            s.apply_prec(xt[r].contiguous(), zr)
            singles.append(zr)
        torch.cuda.synchronize()
        for r in range(3):
            assert torch.equal(zb[r], singles[r])
        b = torch.empty_like(xt)
        s.apply_op(xt, b)
        x1 = torch.empty_like(xt)
        x2 = torch.empty_like(xt)
        st1, i1 = s.solve(b, x1, rtol=1e-10, maxit=40)
        st2, i2 = s.solve(b, x2, rtol=1e-10, maxit=40)
        torch.cuda.synchronize()
        assert st1 == st2 == aao.AAO_OK
        assert torch.equal(x1, x2)
        assert [i["iters"] for i in i1] == [i["iters"] for i in i2]
        assert relerr(x1.cpu().numpy(), x) < 1e-8


def test_initial_guess_and_host_solve():
    p = W.config_2d(N=63, nt=64, alpha=1e-6)
    with aao.Solver(2, p.N, p.nt, p.tau, p.alpha) as s:
        bt = torch.empty((p.nt, p.m), dtype=torch.float64, device=DEV)
        s.build_rhs(cu(p.f), cu(p.psi0), cu(p.psi1), bt)
        x = torch.empty_like(bt)
        st, info = s.solve(bt, x, rtol=1e-10, maxit=50)
        assert st == aao.AAO_OK
        # restarting from the solution converges at once
        x2 = x.clone()
        st, info2 = s.solve(bt, x2, rtol=1e-9, maxit=50, use_x0=True)
        assert st == aao.AAO_OK and info2[0]["iters"] == 0
        # host buffers in, host solution out
        u = np.empty((p.nt, p.m))
        fh = torch.from_numpy(p.f.copy()).pin_memory()
        st, info3 = s.solve_host(fh, p.psi0.copy(), p.psi1.copy(), u, rtol=1e-10, maxit=50)
        assert st == aao.AAO_OK
        assert relerr(u, x.cpu().numpy()) < 1e-12


def test_maxit_reports_not_converged():
    p = W.config_2d(N=63, nt=64, alpha=1e-6)
    with aao.Solver(2, p.N, p.nt, p.tau, p.alpha) as s:
        bt = torch.empty((p.nt, p.m), dtype=torch.float64, device=DEV)
        s.build_rhs(cu(p.f), cu(p.psi0), cu(p.psi1), bt)
        x = torch.empty_like(bt)
        st, info = s.solve(bt, x, rtol=1e-14, maxit=2)
        assert st == aao.AAO_ENOTCONV and info[0]["iters"] == 2


def test_alpha_one_abc_mode():
    """alpha = 1 (ABC preconditioner |C_1|) equals the oracle's fast path, which at
    alpha = 1 is |C_1|^{-1} (pinned densely on the CPU).  At (1D, 63, 64) the smallest
    |Sigma| is about 3e-4 of the largest, far above the 1e-12 singularity threshold, so
    the handle must be created."""
    d, N, nt = 1, 63, 64
    tau = 1.0 / nt
    st, h = aao.aao_create(d, N, nt, tau, 1.0, raw_status=True)
    assert st == aao.AAO_OK, aao.aao_last_error()
    try:
        x = W.random_field((nt, N), seed=700)
        ref = OF.ABACPreconditioner(d, N, nt, tau, 1.0).apply(x)
        xt = cu(x)
        zt = guards.guarded_empty(xt.shape)
        aao.aao_apply_prec(h, xt, zt)
        torch.cuda.synchronize()
        assert relerr(zt.cpu().numpy(), ref) < gates.fp64("prec", d, N, nt, 1.0)
        guards.check(zt)
    finally:
        aao.aao_destroy(h)


@pytest.mark.parametrize("d,N,nt,nrhs", [(1, 63, 64, 1), (2, 63, 128, 3), (3, 63, 64, 2), (2, 255, 256, 1)])
def test_residual_norm_parity(d, N, nt, nrhs):
    """aao_residual_norm == ||b - Y T x|| / ||b|| from the oracle operator, per rhs;
    b = 0 gives the absolute norm."""
    m = N ** d
    tau = 1.0 / nt
    b = W.random_field((nrhs, nt, m), seed=800 + N)
    x = W.random_field((nrhs, nt, m), seed=801 + N) * 1e-3
    if nrhs > 1:
        b[1] = 0.0
    with aao.Solver(d, N, nt, tau, 1e-2, nrhs_max=nrhs) as s:
        rr = torch.empty(nrhs, dtype=torch.float64, device=DEV)
        s.residual_norm(cu(b), cu(x), rr)
        torch.cuda.synchronize()
        got = rr.cpu().numpy()
    for r in range(nrhs):
        res = np.linalg.norm(b[r] - OS.apply_YT(x[r], d, N, tau))
        nb = np.linalg.norm(b[r])
        ref = res / nb if nb > 0 else res
        assert abs(got[r] - ref) <= 1e-13 * ref
