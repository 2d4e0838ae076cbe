"""The bench's CPU FFT restatement of the solve (a throughput reference beside the
oracle) computes the oracle's solution: same iteration count, same solution, true
residual below the tolerance."""
import numpy as np

import bench
import workloads as W
from oracle import fast as OF
from oracle import minres as OM
from oracle import system as OS


def test_scipy_fft_solve_matches_oracle():
    p = W.config_2d(N=31, nt=64, alpha=1e-6, seed=2)
    t, it, xs = bench.scipy_fft_solve(p, 1e-8, 100)
    b = OS.rhs_b(p)
    rel = np.linalg.norm(b - OS.apply_YT(xs, 2, p.N, p.tau)) / np.linalg.norm(b)
    pc = OF.ABACPreconditioner(2, p.N, p.nt, p.tau, p.alpha)
    xo, info = OM.minres(lambda v: OS.apply_YT(v, 2, p.N, p.tau), pc.apply, b, rtol=1e-8, maxit=100)
    assert rel <= 1e-8
    assert it == info["iters"]
    assert np.linalg.norm(xs - xo) / np.linalg.norm(xo) < 1e-10
