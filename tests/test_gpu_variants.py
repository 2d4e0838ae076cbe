"""Every kernel variant computes the same values: the time-pipeline variants (FFT stage
plan x tile x shared-memory layout x load staging, and the small-problem tile) and the
DST variants (stage plan x batched loads, and the small-problem tile), each
against the oracle in FP64 and in FP32, at every supported time length with ragged
mode tails.  The variants only change speed, so each must pass the same gates."""
import os

import numpy as np
import pytest

import gates
import workloads as W
from oracle import fast as OF

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


# (d, N, nt): every time length, mode counts that leave a partial last tile
CASES = [(2, 63, 64), (2, 63, 128), (1, 255, 256), (2, 63, 256), (1, 511, 512), (1, 255, 1024)]
ALPHA = 1e-2


def _time_ref(d, N, nt, x):
    pc = OF.ABACPreconditioner(d, N, nt, 1.0 / nt, ALPHA)
    S = OF.dst_matrix(N)
    return OF.apply_space(pc.apply(OF.apply_space(x, S, d, N)), S, d, N)


@pytest.mark.parametrize("d,N,nt", CASES)
def test_time_variants(d, N, nt, monkeypatch):
    x = W.random_field((nt, N ** d), seed=1700 + nt + N)
    ref = _time_ref(d, N, nt, x)
    tol32 = gates.fp32("time", d, N, nt, ALPHA)
    tol64 = gates.fp64("time", d, N, nt, ALPHA)
    outs = []
    # FP32 on FP64 vectors: 8..15 bulk-staged tile, 16, 17 integer conversions, 18..21
    # loads batched ahead of their conversion, 22, 23 spectral table computed on the fly,
    # 24..29 batched loads with integer conversions of the stores, the loads or both;
    # 30 the one-warp small-problem tile (every precision); 31..33 without the staged
    # table slice
    for v in range(34):
        monkeypatch.setenv("AAO_TIME_VARIANT", f"{v if v == 30 else v & 7},{v}")
        both = v < 8 or v == 30
        for prec in (aao.AAO_PREC_FP64, aao.AAO_PREC_FP32_IR) if both else (aao.AAO_PREC_FP32_IR,):
            with aao.Solver(d, N, nt, 1.0 / nt, ALPHA, precision=prec) as s:
                xt = cu(x)
                yt = torch.empty_like(xt)
                s.apply_time(xt, yt)
                torch.cuda.synchronize()
                y = yt.cpu().numpy()
            if prec == aao.AAO_PREC_FP64:
                assert relerr(y, ref) < tol64, (v, "fp64")
                outs.append(y)
            else:
                assert relerr(y, ref) < tol32, (v, "fp32")
    # the FP64 variants differ only in rounding order
    for y in outs[1:]:
        assert np.abs(y - outs[0]).max() <= 1e-13 * np.abs(outs[0]).max()
    assert aao.aao_wait_timeouts() == 0


@pytest.mark.parametrize("d,N,nt", [(2, 63, 64), (1, 255, 256), (1, 511, 512), (2, 127, 128)])
def test_bulk_staged_time_kernel_guards_and_alignment(d, N, nt, monkeypatch):
    """The bulk-staged FP32 kernels (variants 8..15) and the batched-load ones (18..29)
    write nothing outside their output
    (guard bands at both ends), and a vector that is only 8-byte aligned -- which bulk
    copies cannot address -- is served by the register-staged variant with the same
    gate; every variant's result passes the FP32 gate."""
    import guards
    m = N ** d
    x = W.random_field((nt, m), seed=1750 + nt + N)
    ref = _time_ref(d, N, nt, x)
    tol32 = gates.fp32("time", d, N, nt, ALPHA)
    for v in list(range(8, 16)) + list(range(18, 30)) + [31, 32, 33]:
        monkeypatch.setenv("AAO_TIME_VARIANT", f"3,{v}")
        with aao.Solver(d, N, nt, 1.0 / nt, ALPHA, precision=aao.AAO_PREC_FP32_IR) as s:
            xt = guards.guarded_copy(x)
            yt = guards.guarded_empty(xt.shape)
            s.apply_time(xt, yt)
            torch.cuda.synchronize()
            assert relerr(yt.cpu().numpy(), ref) < tol32, v
            guards.check(yt)
            guards.check(xt)
            # 8-byte aligned views: one double into a larger buffer
            big = torch.zeros(x.size + 2, dtype=torch.float64, device="cuda")
            xv = big[1:1 + x.size].view(nt, m)
            xv.copy_(torch.from_numpy(x))
            outb = torch.zeros(x.size + 2, dtype=torch.float64, device="cuda")
            yv = outb[1:1 + x.size].view(nt, m)
            s.apply_time(xv, yv)
            torch.cuda.synchronize()
            assert relerr(yv.cpu().numpy(), ref) < tol32, (v, "8-byte aligned")
            assert outb[0].item() == 0.0 and outb[-1].item() == 0.0
    assert aao.aao_wait_timeouts() == 0


@pytest.mark.parametrize("d,N,nt", [(2, 63, 64), (2, 127, 64), (2, 255, 64), (2, 511, 64), (3, 63, 64)])
def test_dst_and_prec_variants(d, N, nt, monkeypatch):
    """Both DST stage plans, along every axis, in FP64 (apply_dst) and FP32 (the
    FP32 P_alpha^{-1}, which runs the FP32 DST and the FP32-vector time kernel)."""
    m = N ** d
    x = W.random_field((nt, m), seed=1800 + N + d)
    S = OF.dst_matrix(N)
    ref_dst = OF.apply_space(x, S, d, N)
    ref_prec = OF.ABACPreconditioner(d, N, nt, 1.0 / nt, ALPHA).apply(x)
    tol32 = gates.fp32("prec", d, N, nt, ALPHA)
    for dv in range(9):  # 4..7: interleaved padded layout; 8: the one-warp small-problem tile
        for tv in (1, 5, 30):
            monkeypatch.setenv("AAO_DST_VARIANT", str(dv))
            monkeypatch.setenv("AAO_TIME_VARIANT", f"{tv},{tv}")
            with aao.Solver(d, N, nt, 1.0 / nt, ALPHA) as s:
                xt = cu(x)
                yt = torch.empty_like(xt)
                s.apply_dst(xt, yt)
                torch.cuda.synchronize()
                assert relerr(yt.cpu().numpy(), ref_dst) < 1e-13, (dv, tv)
            with aao.Solver(d, N, nt, 1.0 / nt, ALPHA, precision=aao.AAO_PREC_FP32_IR) as s:
                xt = cu(x)
                zt = torch.empty_like(xt)
                s.apply_prec(xt, zt)
                torch.cuda.synchronize()
                assert relerr(zt.cpu().numpy(), ref_prec) < tol32, (dv, tv)


@pytest.mark.parametrize("d,N,nt,nrhs", [(1, 63, 64, 1), (1, 255, 256, 2), (2, 63, 64, 1), (1, 511, 1024, 1)])
def test_small_problem_tiles_solve(d, N, nt, nrhs, monkeypatch):
    """Small problems take the small tiles by default (one-warp time and DST tiles,
    operator runs of 4 time levels, the small w/x update shape); the solve reaches the
    same true residual as with the standard tiles (AAO_SMALL_TILES=0), checked with the
    oracle's operator, in the same number of iterations (+-1)."""
    from oracle import system as OS
    m = N ** d
    tau = 1.0 / nt
    x = W.random_field((nrhs, nt, m), seed=1900 + N + nt)
    res = {}
    for small in ("1", "0"):
        monkeypatch.setenv("AAO_SMALL_TILES", small)
        with aao.Solver(d, N, nt, tau, 1e-6, nrhs_max=nrhs, graph=True) as s:
            xt = cu(x)
            b = torch.empty_like(xt)
            s.apply_op(xt, b)
            y = torch.empty_like(xt)
            st, info = s.solve(b, y, rtol=1e-10, maxit=100)
            torch.cuda.synchronize()
            assert st == aao.AAO_OK, (small, info)
            res[small] = ([i["iters"] for i in info], b.cpu().numpy(), y.cpu().numpy())
    for small, (it, b, y) in res.items():
        for r in range(nrhs):
            rel = np.linalg.norm(b[r] - OS.apply_YT(y[r], d, N, tau, 1.0)) / np.linalg.norm(b[r])
            assert rel <= 1e-10 * 1.01, (small, r, rel)
    assert all(abs(a - c) <= 1 for a, c in zip(res["1"][0], res["0"][0]))
    assert np.abs(res["1"][2] - res["0"][2]).max() <= 1e-8 * np.abs(res["0"][2]).max()
    assert aao.aao_wait_timeouts() == 0
