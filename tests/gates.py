"""Parity gates for the preconditioner kernels, from a rounding-error model.

Model (relative max-norm error of one application against the oracle):

    err  <~  u * ( a * L  +  b * log2(n) * alpha^{-(n-1)/n}  [+ c * R] )

* u: unit round-off of the arithmetic (2^-24 FP32, 2^-47 for the double-word
  operations, 2^-53 FP64).
* a * L: the transforms.  A radix-r FFT or DST of length L with accurately rounded
  twiddles has relative error O(u log2 L); L sums log2 of the lengths the kernel path
  applies: the time pipeline (log2 n) and, for P_alpha^{-1}, two DST passes per
  spatial axis (2 d log2(N+1)).
* b * log2(n) * alpha^{-(n-1)/n}: the alpha-scaling.  The pipeline ends with D_alpha^{-1},
  which multiplies time level t by alpha^{-t/n} (up to alpha^{-(n-1)/n} at the last
  level), so the rounding errors of the scaled transforms are amplified at late time
  levels relative to the entries that set the max norm (the paper's closing remark of
  Section 2.3: small alpha costs accuracy in floating point).
* c * R (FP64 comparisons only): the oracle's own rounding.  It applies explicit DFT
  (n x n) and DST ((N) x (N)) matrices by matrix products, whose error grows like
  u sqrt(length) per product; R = sqrt(n) + (oracle DST passes) * sqrt(N+1).

The constants a, b, c were fitted per arithmetic to the errors measured on GB300 over
every parity case of the test suite (dimensions 1-3, n = 64..1024, alpha = 1e-1..1e-6),
then scaled so that the largest gate-to-error ratio over those cases is 30; the
smallest is 9.7 (FP32), 7.7 (double-word pipeline), 6.8 (double-word DST) and 2.5
(FP64, whose errors scatter more because the oracle's own rounding is of the same
order).  FP64 gates are additionally capped by the specification: 1e-12 relative for
alpha >= 1e-3 and 1e-9 at alpha = 1e-6.
"""
import math

U32 = 2.0 ** -24
UDW = 2.0 ** -47
U64 = 2.0 ** -53


def amp(alpha, n):
    """alpha^{-(n-1)/n}: the largest entry of D_alpha^{-1}."""
    return alpha ** (-(n - 1) / n)


def transform_logs(kind, d, N, n):
    ln, lm = math.log2(n), math.log2(N + 1)
    return {"prec": ln + 2 * d * lm, "time": ln, "dst": d * lm}[kind]


def fp32(kind, d, N, n, alpha):
    """FP32/complex64 preconditioner pipeline (kind 'prec' = P_alpha^{-1}, 'time' = its time part)."""
    return U32 * (10.0 * transform_logs(kind, d, N, n) + 0.3 * math.log2(n) * amp(alpha, n))


def dword(kind, d, N, n, alpha=1.0):
    """Double-word (pairs of FP32) pipeline; kind 'dst' = the DST alone (no alpha term)."""
    if kind == "dst":
        return UDW * 8.0 * transform_logs("dst", d, N, n)
    return UDW * (3.4 * transform_logs(kind, d, N, n) + 0.115 * math.log2(n) * amp(alpha, n))


def fp64(kind, d, N, n, alpha, oracle_dst_passes=None):
    """FP64 pipeline against the FP64 oracle, capped by the specification."""
    if oracle_dst_passes is None:
        oracle_dst_passes = {"prec": 2 * d, "time": 4 * d}[kind]
    model = U64 * (26.0 * transform_logs(kind, d, N, n) + 0.28 * math.log2(n) * amp(alpha, n)
                   + 8.5 * (math.sqrt(n) + oracle_dst_passes * math.sqrt(N + 1)))
    spec = 1e-12 if alpha >= 1e-3 else 1e-9
    return min(spec, model)
