"""The allocation-free residual entry point agrees with the handle-based one.

aao_residual_norm_noalloc serves callers that cannot allocate device memory when
they need a residual check (a host framework's pool allocator owns all device
memory, or cudaMalloc's implicit synchronisation is not acceptable in their
loop).  It keeps its partial sums in a static device array instead of a handle's
workspace; this test calls it through the C ABI twice in a row and compares both
results with aao_residual_norm on the same inputs.  The file name makes pytest
collect it last.
"""
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
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    aao.lib()


@pytest.mark.parametrize("d,N,nt,nrhs,c2,zero_b", [(1, 63, 64, 1, 1.0, False), (2, 63, 128, 3, 1.0, False),
                                                   (3, 63, 64, 2, 1.0, False), (2, 255, 256, 1, 1.0, False),
                                                   (2, 127, 64, 2, 2.7, False), (1, 127, 128, 2, 0.6, True)])
def test_noalloc_matches_handle_entry_point(d, N, nt, nrhs, c2, zero_b):
    """Two calls in a row agree with aao_residual_norm; with a wave speed c2 != 1 the
    operator's coefficient follows c2; with b = 0 both return the absolute norm."""
    m = N ** d
    tau = 1.0 / nt
    b = torch.from_numpy(W.random_field((nrhs, nt, m), seed=900 + N)).cuda()
    if zero_b:
        b.zero_()
    x = torch.from_numpy(W.random_field((nrhs, nt, m), seed=901 + N) * 1e-3).cuda()
    with aao.Solver(d, N, nt, tau, 1e-2, c2=c2, nrhs_max=nrhs) as s:
        ref = torch.empty(nrhs, dtype=torch.float64, device="cuda")
        s.residual_norm(b, x, ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
    assert np.all(ref > 0)
    for _ in range(2):
        got = torch.full((nrhs,), -1.0, dtype=torch.float64, device="cuda")
        aao.aao_residual_norm_noalloc(d, N, nt, tau, b, x, got, nrhs, c2=c2)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref)), (got, ref)


def test_noalloc_later_calls_allocate_nothing():
    """After the first call on the device (which may load the library's module), the
    device's free memory stays the same across further calls."""
    d, N, nt, nrhs = 2, 63, 64, 2
    m = N ** d
    b = torch.from_numpy(W.random_field((nrhs, nt, m), seed=950)).cuda()
    x = torch.from_numpy(W.random_field((nrhs, nt, m), seed=951)).cuda()
    outs = [torch.empty(nrhs, dtype=torch.float64, device="cuda") for _ in range(5)]
    aao.aao_residual_norm_noalloc(d, N, nt, 1.0 / nt, b, x, outs[0], nrhs)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for o in outs[1:]:
        aao.aao_residual_norm_noalloc(d, N, nt, 1.0 / nt, b, x, o, nrhs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    first = outs[0].cpu().numpy()
    for o in outs[1:]:
        assert np.array_equal(o.cpu().numpy(), first)


def test_noalloc_rejects_too_many_rhs():
    x = torch.zeros((65, 64, 63), dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    st = aao.aao_residual_norm_noalloc(1, 63, 64, 1 / 64, x, x, out, 65, raw_status=True)
    assert st == aao.AAO_EINVAL
    assert "nrhs" in aao.lib().aao_noalloc_last_error().decode()
