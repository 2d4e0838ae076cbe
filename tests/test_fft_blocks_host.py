"""CPU checks of the in-register DFT building blocks of the FFT engine (fft_smem.cuh):
the 16-point DFT with its internal twiddles folded into multiply-adds, its inverse by
the real/imaginary swap, and the first-stage DFTs that apply a real diagonal scaling
to their inputs.  The header's host-callable templates are compiled with nvcc for the
host and compared with numpy.fft on seeded inputs (double within 1e-15, float within
the FP32 rounding of a 16-point transform)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_03574_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include "fft_smem.cuh"
using namespace aao;
template <typename C> void run(int kind, int n) {
  using R = decltype(C::x);
  for (int t = 0; t < n; ++t) {
    C v[16]; R s[16];
    for (int i = 0; i < 16; ++i) { double a, b; if (scanf("%lf %lf", &a, &b) != 2) return; v[i].x = (R)a; v[i].y = (R)b; }
    for (int i = 0; i < 16; ++i) { double a; if (scanf("%lf", &a) != 1) return; s[i] = (R)a; }
    if (kind == 0) dft16_fma<false>(v);
    else if (kind == 1) dft16_fma<true>(v);
    else if (kind == 2) dft_r_scaled<16>(v, s);
    else dft_r_scaled<4>(v, s);
    const int len = kind == 3 ? 4 : 16;
    for (int i = 0; i < len; ++i) printf("%.17g %.17g\n", (double)v[i].x, (double)v[i].y);
  }
}
int main(int argc, char** argv) {
  const int kind = argv[1][0] - '0', fp32 = argv[2][0] - '0', n = 64;
  if (fp32) run<float2>(kind, n); else run<double2>(kind, n);
  return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("fftblocks")
    src = d / "blocks.cu"
    src.write_text(PROG)
    exe = d / "blocks"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), "-x", "cu", str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    return str(exe)


def _run(exe, kind, fp32, v, s):
    lines = []
    for t in range(v.shape[0]):
        lines += [f"{a.real:.17g} {a.imag:.17g}" for a in v[t]]
        lines += [f"{a:.17g}" for a in s[t]]
    out = subprocess.run([exe, str(kind), str(fp32)], input="\n".join(lines), capture_output=True,
                         text=True, check=True).stdout.split()
    z = np.array(out, dtype=np.float64).reshape(v.shape[0], -1, 2)
    return z[..., 0] + 1j * z[..., 1]


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_dft_blocks_match_numpy(prog, kind, fp32):
    rng = np.random.default_rng(900 + 10 * kind + fp32)
    v = rng.standard_normal((64, 16)) + 1j * rng.standard_normal((64, 16))
    s = rng.uniform(0.01, 3.0, (64, 16))
    if fp32:  # the program sees the inputs rounded to float
        v = v.astype(np.complex64).astype(np.complex128)
        s = s.astype(np.float32).astype(np.float64)
    got = _run(prog, kind, fp32, v, s)
    if kind == 0:
        ref = np.fft.fft(v, axis=1)
    elif kind == 1:
        ref = np.fft.ifft(v, axis=1) * 16  # unnormalised inverse
    elif kind == 2:
        ref = np.fft.fft(v * s, axis=1)
    else:
        ref = np.fft.fft(v[:, :4] * s[:, :4], axis=1)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < (2e-6 if fp32 else 1e-15), err
