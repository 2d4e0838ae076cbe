"""Small profiling driver for ncu captures: runs `--reps` preconditioner
applications (or full solves) of one problem size through the C ABI.

  python -m paper_2306_03574_gb300.profile_case --d 2 --N 255 --nt 256 --what prec --reps 1
"""
from __future__ import annotations

import argparse
import os

import numpy as np
import torch

from . import aao


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--N", type=int, default=255)
    ap.add_argument("--nt", type=int, default=256)
    ap.add_argument("--alpha", type=float, default=1e-6)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--precision", choices=["fp64", "fp32", "f32x2"], default="fp64")
    ap.add_argument("--what", choices=["prec", "time", "dst", "op", "solve"], default="prec")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--time-variant", type=int, default=None, help="time-kernel variant 0..7")
    ap.add_argument("--dst-variant", type=int, default=None, help="DST variant 0..1")
    a = ap.parse_args()
    if a.time_variant is not None:
        os.environ["AAO_TIME_VARIANT"] = f"{a.time_variant},{a.time_variant},{a.time_variant}"
    if a.dst_variant is not None:
        os.environ["AAO_DST_VARIANT"] = str(a.dst_variant)
    prec = {"fp64": aao.AAO_PREC_FP64, "fp32": aao.AAO_PREC_FP32_IR, "f32x2": aao.AAO_PREC_F32X2}[a.precision]
    m = a.N ** a.d
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal((a.nrhs, a.nt, m))).cuda()
    y = torch.empty_like(x)
    with aao.Solver(a.d, a.N, a.nt, 1.0 / a.nt, a.alpha, precision=prec, nrhs_max=a.nrhs) as s:
        for _ in range(a.reps):
            if a.what == "prec":
                s.apply_prec(x, y)
            elif a.what == "time":
                s.apply_time(x, y)
            elif a.what == "dst":
                s.apply_dst(x, y)
            elif a.what == "op":
                s.apply_op(x, y)
            else:
                s.apply_op(x, y)
                st, info = s.solve(y, x, rtol=1e-8, maxit=50)
                assert st == aao.AAO_OK, info
        torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
