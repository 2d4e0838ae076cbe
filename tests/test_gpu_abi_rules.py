"""The C ABI's allocation and synchronisation rules: aao_create reserves every buffer
a later call needs (the FP32 buffer of aao_apply_prec; with opts.host_staging the
buffers of aao_solve_host), and creating a handle does not wait for work that another
stream has in flight."""
import time

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


def test_workspace_fixed_at_create():
    d, N, nt = 2, 63, 64
    p = W.config_2d(N=N, nt=nt, alpha=1e-3)
    with aao.Solver(d, N, nt, p.tau, p.alpha, precision=aao.AAO_PREC_FP32_IR) as s:
        w0 = s.workspace_bytes
        x = torch.from_numpy(W.random_field((nt, p.m), seed=5)).cuda()
        z = torch.empty_like(x)
        s.apply_prec(x, z)
        torch.cuda.synchronize()
        assert s.workspace_bytes == w0
    for prec in (aao.AAO_PREC_FP64, aao.AAO_PREC_F32X2, aao.AAO_PREC_FP32_IR):
        with aao.Solver(d, N, nt, p.tau, 1e-3, precision=prec, host_staging=True, graph=True) as s:
            w0 = s.workspace_bytes
            u = np.empty((nt, p.m))
            st, info = s.solve_host(p.f, p.psi0, p.psi1, u, rtol=1e-8, maxit=200)
            assert st == aao.AAO_OK, info
            assert s.workspace_bytes == w0, prec
    # without the option the first host-buffer solve reserves its buffers (documented)
    with aao.Solver(d, N, nt, p.tau, 1e-3) as s:
        w0 = s.workspace_bytes
        u = np.empty((nt, p.m))
        s.solve_host(p.f, p.psi0, p.psi1, u, rtol=1e-8, maxit=200)
        assert s.workspace_bytes > w0


def test_create_does_not_wait_for_other_streams():
    d, N, nt = 2, 127, 128
    aao.Solver(d, N, nt, 1.0 / nt, 1e-6).close()  # kernels loaded, allocator warm
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    done = torch.cuda.Event()
    with torch.cuda.stream(side):
        torch.cuda._sleep(int(1.5e9))  # a bounded spin of about 0.75 s at 2 GHz
        done.record(side)
    t0 = time.perf_counter()
    s = aao.Solver(d, N, nt, 1.0 / nt, 1e-6)
    t1 = time.perf_counter()
    still_running = not done.query()
    side.synchronize()
    t2 = time.perf_counter()
    s.close()
    assert still_running, "aao_create returned only after the other stream's kernel ended"
    assert t1 - t0 < 0.5 * (t2 - t0), (t1 - t0, t2 - t0)
