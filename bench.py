"""Benchmark: FP64 ABAC-preconditioned MINRES solves of the 2D wave workload.

Workload (one "step" = one full solve of the hot path): 2D wave u_tt = Lap u + f on
[0,1]^2, 5-point Laplacian on a 255 x 255 interior grid, 256 time levels, T = 1,
manufactured u = sin(pi x) sin(pi y) cos(sqrt(2) pi t) with seeded U[-1,1]*1e-3 source
noise (16,646,400 unknowns), alpha = 1e-6, MINRES from a zero guess to a TRUE
relative residual of 1e-8; each step builds b = Y f from the resident inputs
(f, psi0, psi1 already in HBM) and solves.  FP64 end to end.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas (one problem
per GPU, no data-path collective; weak scaling) under torch.distributed.run.
--impl reference times the CPU oracle (the paper's method written plainly in
NumPy) on the same workload: each step is a bounded sample, one MINRES
iteration's operator work (one P_alpha^{-1} application and two Y T
applications), scaled to solves/s by the oracle's own iteration count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("MINRES solves/s & unknown·iters/s at rel-res 1e-8; "
          "precond-apply HBM GB/s vs 8 TB/s")
# Named workloads.  The default is the FP64 2D one; the others are the mixed-precision
# and batched rows (run explicitly with --workload).  The mixed-precision rows take
# alpha = 1e-3: the FP32 preconditioner's round-off grows like alpha^{-(n-1)/n}, and
# 1e-3 balances it against the preconditioner's approximation error (measured sweep).
WORKLOADS = {
    "2d255_fp64": dict(d=2, N=255, nt=256, alpha=1e-6, rtol=1e-8, maxit=100, seed=2, nrhs=1,
                       precision="fp64"),
    "1d63_fp64": dict(d=1, N=63, nt=64, alpha=1e-6, rtol=1e-8, maxit=100, seed=1, nrhs=1,
                      precision="fp64"),
    "2d511_fp64": dict(d=2, N=511, nt=512, alpha=1e-6, rtol=1e-8, maxit=100, seed=3, nrhs=1,
                       precision="fp64"),
    "2d511_mixed": dict(d=2, N=511, nt=512, alpha=1e-3, rtol=1e-8, maxit=200, seed=3, nrhs=1,
                        precision="fp32"),
    "2d255_mixed": dict(d=2, N=255, nt=256, alpha=1e-3, rtol=1e-8, maxit=200, seed=2, nrhs=1,
                        precision="fp32"),
    "3d127x8_mixed": dict(d=3, N=127, nt=128, alpha=1e-3, rtol=1e-8, maxit=200, seed=4, nrhs=8,
                          precision="fp32"),
    "3d127x8_fp64": dict(d=3, N=127, nt=128, alpha=1e-6, rtol=1e-8, maxit=100, seed=4, nrhs=8,
                         precision="fp64"),
    # Example 2's variable coefficient a = (30 + sin^2 x)(30 + sin^2 y), mean-coefficient preconditioner
    "2d255_varcoef_fp64": dict(d=2, N=255, nt=256, alpha=1e-6, rtol=1e-8, maxit=200, seed=0, nrhs=1,
                               precision="fp64", varcoef=True),
    "2d255_varcoef_mixed": dict(d=2, N=255, nt=256, alpha=1e-3, rtol=1e-8, maxit=300, seed=0, nrhs=1,
                                precision="fp32", varcoef=True),
    # double-float time pipeline (pairs of FP32 numbers on the FP32 pipes), FP64 elsewhere
    "2d255_f32x2": dict(d=2, N=255, nt=256, alpha=1e-6, rtol=1e-8, maxit=100, seed=2, nrhs=1,
                        precision="f32x2"),
    "2d511_f32x2": dict(d=2, N=511, nt=512, alpha=1e-6, rtol=1e-8, maxit=100, seed=3, nrhs=1,
                        precision="f32x2"),
    "3d127x8_f32x2": dict(d=3, N=127, nt=128, alpha=1e-6, rtol=1e-8, maxit=100, seed=4, nrhs=8,
                          precision="f32x2"),
}
# FP32 operations per FP64-equivalent flop of the double-word arithmetic: a sloppy
# double-word addition takes 11 FP32 flops (2Sum 6, low-part sum 1, fold-in 1,
# Fast2Sum 3), a double-word product 10 (product 1, three FMAs 6, Fast2Sum 3); an FFT's
# flop count is 60 % additions and 40 % multiplications (radix-2 butterfly: 6 + 4).
DW_FP32_FLOPS_PER_FLOP = 0.6 * 11 + 0.4 * 10
WORKLOAD = dict(WORKLOADS["2d255_fp64"])
WORKLOAD_NAME = ["2d255_fp64"]
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def log2(v):
    return v.bit_length() - 1


def algorithmic_flops(cls: str, d: int, N: int, nt: int, unknowns: int, varcoef: bool = False) -> float:
    """Algorithmic FLOPs of one launch of a kernel class (standard FFT count
    5 L log2 L per complex transform of length L, i.e. 2.5 L log2 L per real one)."""
    M = N + 1
    if cls.startswith("time"):
        # 4 real transforms of length n, two spectral multiplies (6 flops per complex
        # value = 6 per real unknown), three diagonal scalings
        return unknowns * (4 * 2.5 * log2(nt) + 6 + 3)
    if cls.startswith("dst"):
        # DST-I of length N counted as one real transform of length N+1
        return unknowns * 2.5 * log2(M)
    if cls == "yt_resvec":
        # refinement residual in the DST basis: the operator (4), b minus it (1), its
        # square accumulated (2)
        return unknowns * 7
    if cls.startswith("yt"):
        # Y T v per unknown.  With a constant coefficient, MINRES runs in the DST basis,
        # where the operator is Lambda (v_i + v_{i-2}) - 2 v_{i-1} (4 flops); the
        # physical residual check applies the stencil L (2d neighbours summed, scaled
        # and subtracted from the scaled centre: 2d + 2) and the time band (3).  The
        # variable-coefficient L, the centre plus 2d face-weighted differences with
        # time-invariant weights, takes a difference and a multiply-add per face (6d)
        # per application, plus the time band.  A fused dot adds 2, a residual 3.
        if varcoef:
            op = 6 * d + 3
        elif cls == "yt_res":
            op = 2 * d + 5
        else:
            op = 4
        return unknowns * (op + (2 if cls == "yt_dot" else 3 if cls == "yt_res" else 0))
    if cls == "wx_res":
        # w and x updates (3 + 2 multiply-adds, one product: 7) and the DST-basis
        # residual Lambda (x_i + x_{i-2}) - 2 x_{i-1}, its difference from b and its
        # square accumulated (7)
        return unknowns * 14
    return 0.0


def algorithmic_bytes(cls: str, d: int, N: int, nt: int, unknowns: int, vec_bytes: int) -> float:
    """Bytes one launch must move at least: its vectors in and out once (vec_bytes per
    element: 8 for FP64 vectors, 4 for FP32 ones) plus, for the time kernel, the
    spectral table A_k, B_k (k = 0..n/2, one entry pair per mode pair, shared by all
    right-hand sides)."""
    m = N ** d
    if cls.startswith("time"):
        csize = 8 if cls == "time_f32" else 16
        return 2 * vec_bytes * unknowns + (nt // 2 + 1) * ((m + 1) // 2) * 2 * csize
    if cls.startswith("dst"):
        return 2 * vec_bytes * unknowns
    if cls in ("yt", "yt_dot", "yt_res"):
        # one vector in and one out (the fused dot's operand is the input itself; the
        # residual reads b instead of writing)
        return 16 * unknowns
    if cls == "yt_resvec":
        # reads x and b, writes r
        return 24 * unknowns
    if cls == "wx_res":
        # reads z, w_{j-1}, w_j, x, b; writes w_{j+1}, x
        return 56 * unknowns
    return 0.0


_ALU_PEAKS = {}


def alu_peaks_measured():
    """FP64 (DFMA) and FP32 (FFMA) rates of the library's FMA-loop probe on this GPU,
    measured once per process (outside any timed region)."""
    if not _ALU_PEAKS:
        try:
            import paper_2306_03574_gb300 as aao
            f64, ms64 = aao.aao_alu_peak(aao.AAO_PREC_FP64, 1 << 14)
            f32, ms32 = aao.aao_alu_peak(aao.AAO_PREC_FP32_IR, 1 << 18)
            _ALU_PEAKS.update(fp64_tflops=f64, fp32_tflops=f32, fp64_ms=ms64, fp32_ms=ms32,
                              how="aao_alu_peak: 8 blocks x 256 threads per SM, 8 independent FMA chains "
                                  "per thread, best of 3 CUDA-event timings")
        except Exception as e:  # statistics only
            _ALU_PEAKS["error"] = repr(e)[:200]
    return dict(_ALU_PEAKS)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0, period_ms: int = 50):
        self.proc = None
        self.path = None
        self.index = index
        self.period = period_ms

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", f"-lms", str(self.period)],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(rows)}


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(cls: str, variant=None):
    """ncu DRAM bytes per launch for the dominant kernel, if captured for the current
    kernel source and the kernel variant the bench runs (profiles/traffic.json,
    written from an ncu capture)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    r = rec.get(cls)
    if not r:
        return None
    srcs = [os.path.join(ROOT, "paper_2306_03574_gb300", "csrc", f) for f in r.get("sources", [])]
    try:
        if source_hash(srcs) != r.get("source_hash"):
            return None
    except Exception:
        return None
    if variant is not None and r.get("variant") is not None and r["variant"] != variant:
        return None
    if WORKLOAD_NAME[0] not in r.get("workloads", [r.get("workload")]):
        return None
    return r.get("bytes_per_launch")


def dist_setup(n_gpus: int, backend: str):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def reduce_max(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_problem():
    import workloads as W
    from oracle import fast as OF
    from oracle import system as OS
    p = W.config_2d(N=WORKLOAD["N"], nt=WORKLOAD["nt"], alpha=WORKLOAD["alpha"], seed=WORKLOAD["seed"])
    pc = OF.ABACPreconditioner(2, p.N, p.nt, p.tau, p.alpha)
    A = lambda v: OS.apply_YT(v, 2, p.N, p.tau)
    return p, pc, A


def oracle_full_solve(p, pc, A):
    """One full oracle solve (rhs + MINRES to true rel-res 1e-8); returns (seconds, iters)."""
    from oracle import minres as OM
    from oracle import system as OS
    t0 = time.perf_counter()
    b = OS.rhs_b(p)
    x, info = OM.minres(A, pc.apply, b, rtol=WORKLOAD["rtol"], maxit=WORKLOAD["maxit"])
    return time.perf_counter() - t0, info["iters"]


def oracle_iteration_sample(p, pc, A, v):
    """One MINRES iteration's operator work of the oracle: P^{-1} v, Y T z, Y T x."""
    t0 = time.perf_counter()
    z = pc.apply(v)
    A(z)
    A(v)
    return time.perf_counter() - t0


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import numpy as np
    p, pc, A = oracle_problem()
    from oracle import system as OS
    v = OS.rhs_b(p)
    # warm-up: the first one is a full oracle solve, which also gives the iteration count
    t_full, iters = oracle_full_solve(p, pc, A)
    for _ in range(max(0, args.warmup - 1)):
        oracle_iteration_sample(p, pc, A, v)
    ts = [oracle_iteration_sample(p, pc, A, v) for _ in range(args.steps)]
    t_step = float(np.mean(ts))
    # a solve = rhs + one P^{-1} at start + iters x (P^{-1} + 2 Y T): ~ (iters + 1) samples
    t_solve = t_step * (iters + 1)
    value = 1.0 / t_solve
    cores = os.cpu_count()
    unknowns = p.nt * p.m
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(unknowns),
        "iters_per_solve": iters, "unknown_iters_per_s": unknowns * iters / t_solve,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step one oracle MINRES iteration's operator work at full size "
                                   f"(1 P^-1 + 2 YT), scaled by (iters+1)={iters + 1}; one full oracle "
                                   f"solve in warm-up took {t_full:.2f} s"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(unknowns, name=None):
    W_ = WORKLOAD
    vec_mb = unknowns * 8 / 1e6
    return {"workload": f"{W_['d']}d_wave_N{W_['N']}_nt{W_['nt']}_x{W_['nrhs']}_{W_['precision']}"
                        f"_minres_relres{W_['rtol']:g}",
            "name": name or "2d255_fp64", "d": W_["d"], "N": W_["N"], "nt": W_["nt"],
            "unknowns": unknowns, "alpha": W_["alpha"], "rtol": W_["rtol"], "rhs": W_["nrhs"],
            "precision": W_["precision"], "seed": W_["seed"],
            "l2": f"inputs larger than L2: every vector is {vec_mb:.0f} MB per rhs (L2 126 MB)",
            "parallelism": "replicas (one independent problem per GPU)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def error_vs_exact(x_host, p):
    """E = max_k h^{d/2} ||u^(k) - u(x, k tau)||_2 over the time levels (the error
    measure of the paper's Section 3), for problems with a known exact solution."""
    import numpy as np
    if p.exact is None:
        return None
    h = 1.0 / (p.N + 1)
    worst = 0.0
    for k in range(p.nt):
        diff = x_host[k] - p.exact((k + 1) * p.tau)
        worst = max(worst, float(h ** (p.d / 2.0) * np.linalg.norm(diff)))
    return worst


def scipy_fft_solve(p, rtol, maxit):
    """The same solve restated for the host cores with scipy.fft (FFT-based DSTs and
    time transforms on all cores, NumPy elementwise work): DST of b, preconditioned
    MINRES in the DST basis stopping on the true relative residual, DST back.  A fair
    CPU-throughput reference beside the oracle (which applies explicit DFT and DST
    matrices); not part of the product.  Returns (seconds, iterations, solution)."""
    import math
    import numpy as np
    import scipy.fft as sf
    w = os.cpu_count()
    d, N, n, tau, alpha, c2 = p.d, p.N, p.nt, p.tau, p.alpha, p.c2
    m = N ** d
    h = 1.0 / (N + 1)
    axes = tuple(range(1, d + 1))
    t0 = time.perf_counter()

    def U(v):
        return sf.dstn(v.reshape((n,) + (N,) * d), type=1, axes=axes, norm="ortho",
                       workers=w).reshape(n, m)

    mu1 = 4.0 / (h * h) * np.sin(np.arange(1, N + 1) * np.pi * h / 2.0) ** 2
    mu = np.zeros((N,) * d)
    for a in range(d):
        shp = [1] * d
        shp[d - 1 - a] = N
        mu = mu + mu1.reshape(shp)
    lm1 = (0.5 * c2 * tau * tau * mu).ravel()
    lam = 1.0 + lm1
    k = np.arange(n // 2 + 1)[:, None]
    a_ = math.exp(math.log(alpha) / n)
    th = np.exp(2j * np.pi * k / n)
    G = ((1 - a_ * th) ** 2 + lm1[None, :] * (1 + a_ * a_ * th * th)) ** -0.5
    t = np.arange(n)[:, None]
    dinv = alpha ** (-t / n)
    d2 = alpha ** (2.0 * t / n)

    def prec(v):
        z = sf.irfft(G * sf.rfft(v * dinv, axis=0, workers=w), n=n, axis=0, workers=w)
        z = sf.irfft(np.conj(G) * sf.rfft(z * d2, axis=0, workers=w), n=n, axis=0, workers=w)
        return z * dinv

    def A(v):  # Y T in the DST basis: slot n-1-i holds lam (v_i + v_{i-2}) - 2 v_{i-1}
        T = lam * v
        T[1:] -= 2.0 * v[:-1]
        T[2:] += lam * v[:-2]
        return T[::-1].copy()

    # right-hand side (first blocks tau^2 f0/2 + tau psi1 + psi0 and tau^2 f1 - L psi0)
    F = tau * tau * np.asarray(p.f, dtype=np.float64)
    F[0] = tau * tau * p.f[0] / 2.0 + tau * p.psi1 + p.psi0
    def U1(v):  # one time level
        return sf.dstn(v.reshape((N,) * d), type=1, norm="ortho", workers=w).ravel()

    Lpsi0 = U1(lam * U1(np.asarray(p.psi0, dtype=np.float64)))
    F[1] = tau * tau * p.f[1] - Lpsi0
    b = U(F[::-1].copy())
    bn = np.linalg.norm(b)
    # preconditioned MINRES (Lanczos on P^{-1}, Givens QR), x0 = 0
    x = np.zeros_like(b)
    v = b.copy()
    z = prec(v)
    gam = math.sqrt(float(np.vdot(z, v)))
    gam_prev = 1.0
    v_prev = np.zeros_like(b)
    w_, w_prev = np.zeros_like(b), np.zeros_like(b)
    eta, c, c_prev, s_, s_prev = gam, 1.0, 1.0, 0.0, 0.0
    it = 0
    while it < maxit:
        zn = z / gam
        Az = A(zn)
        delta = float(np.vdot(Az, zn))
        vn = Az - (delta / gam) * v - (gam / gam_prev) * v_prev
        znew = prec(vn)
        gnew = math.sqrt(max(float(np.vdot(znew, vn)), 0.0))
        a0 = c * delta - c_prev * s_ * gam
        a1 = math.hypot(a0, gnew)
        a2 = s_ * delta + c_prev * c * gam
        a3 = s_prev * gam
        cn, sn = a0 / a1, gnew / a1
        wn = (zn - a3 * w_prev - a2 * w_) / a1
        x += cn * eta * wn
        eta = -sn * eta
        w_prev, w_ = w_, wn
        v_prev, v = v, vn
        z, gam_prev, gam = znew, gam, gnew
        c_prev, c, s_prev, s_ = c, cn, s_, sn
        it += 1
        if np.linalg.norm(b - A(x)) / bn <= rtol:
            break
    xs = U(x)
    return time.perf_counter() - t0, it, xs


def cufft_comparison(s, p, dev, reps=10):
    """The time part of P_alpha^{-1} written with torch.fft (cuFFT) and torch elementwise
    kernels: D^{-1}, rfft, x G, irfft, D^2, rfft, x conj(G), irfft, D^{-1} along time for
    every DST mode, G = Sigma^{-1/2} on bins k = 0..n/2.  A library baseline for the
    fused kernel (timed the same way on the same data), not part of the product."""
    import math
    import torch
    d, N, n, tau, alpha, c2 = p.d, p.N, p.nt, p.tau, p.alpha, p.c2
    m = N ** d
    f64, c128 = torch.float64, torch.complex128
    h = 1.0 / (N + 1)
    j = torch.arange(1, N + 1, dtype=f64, device=dev)
    mu1 = 4.0 / (h * h) * torch.sin(j * math.pi * h / 2.0) ** 2
    mu = torch.zeros((N,) * d, dtype=f64, device=dev)
    for a in range(d):
        shp = [1] * d
        shp[d - 1 - a] = N
        mu = mu + mu1.reshape(shp)
    lm1 = (0.5 * c2 * tau * tau * mu).reshape(1, m)
    k = torch.arange(n // 2 + 1, dtype=f64, device=dev).reshape(-1, 1)
    la = math.log(alpha) / n
    a = math.exp(la)
    th = torch.exp(1j * (2 * math.pi / n) * k.to(c128))
    sig = (1 - a * th) ** 2 + lm1.to(c128) * (1 + a * a * th * th)
    G = sig ** -0.5
    t = torch.arange(n, dtype=f64, device=dev).reshape(-1, 1)
    dinv = alpha ** (-t / n)
    d2 = alpha ** (2 * t / n)
    x = torch.randn((n, m), dtype=f64, device=dev, generator=torch.Generator(device=dev).manual_seed(7))

    def pipe(v):
        z = torch.fft.irfft(G * torch.fft.rfft(v * dinv, dim=0), n=n, dim=0)
        z = torch.fft.irfft(G.conj() * torch.fft.rfft(z * d2, dim=0), n=n, dim=0)
        return z * dinv

    ours = torch.empty_like(x)
    for _ in range(3):
        ref = pipe(x)
        s.apply_time(x, ours)
    torch.cuda.synchronize(dev)
    diff = float((ref - ours).abs().max() / ref.abs().max())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        pipe(x)
    e1.record()
    torch.cuda.synchronize(dev)
    t_lib = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        s.apply_time(x, ours)
    e1.record()
    torch.cuda.synchronize(dev)
    t_ours = e0.elapsed_time(e1) / reps
    return {"time_pipeline_ms_cufft": t_lib, "time_pipeline_ms_fused_kernel": t_ours,
            "speedup": t_lib / t_ours, "max_rel_diff": diff,
            "note": "torch.fft (cuFFT) rfft/irfft along time + torch elementwise kernels, FP64, "
                    "same shape; CUDA events, mean of %d" % reps}



def run_gpu(args, world, rank, local, emit=True):
    import numpy as np
    import torch

    import paper_2306_03574_gb300 as aao
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    d, N, nt, nrhs = WORKLOAD["d"], WORKLOAD["N"], WORKLOAD["nt"], WORKLOAD["nrhs"]
    seed = WORKLOAD["seed"] + 1000 * rank
    varcoef = WORKLOAD.get("varcoef", False)
    if d == 3:
        p, fb = W.config_3d_batched(N=N, nt=nt, nrhs=nrhs, seed=seed, alpha=WORKLOAD["alpha"])
        fnp = fb
        p0np = np.zeros((nrhs, p.m))
        p1np = np.zeros((nrhs, p.m))
    elif d == 1:
        p = W.config_1d(N=N, nt=nt, alpha=WORKLOAD["alpha"], seed=seed)
        fnp = np.broadcast_to(p.f, (nrhs,) + p.f.shape).copy()
        p0np = np.broadcast_to(p.psi0, (nrhs, p.m)).copy()
        p1np = np.broadcast_to(p.psi1, (nrhs, p.m)).copy()
    elif varcoef:
        p = W.example2(N, nt, alpha=WORKLOAD["alpha"])
        fnp = np.broadcast_to(p.f, (nrhs,) + p.f.shape).copy()
        p0np = np.broadcast_to(p.psi0, (nrhs, p.m)).copy()
        p1np = np.broadcast_to(p.psi1, (nrhs, p.m)).copy()
    else:
        p = W.config_2d(N=N, nt=nt, alpha=WORKLOAD["alpha"], seed=seed)
        fnp = np.broadcast_to(p.f, (nrhs,) + p.f.shape).copy()
        p0np = np.broadcast_to(p.psi0, (nrhs, p.m)).copy()
        p1np = np.broadcast_to(p.psi1, (nrhs, p.m)).copy()
    unknowns = p.nt * p.m * nrhs
    f = torch.from_numpy(fnp).to(dev)
    psi0 = torch.from_numpy(p0np).to(dev)
    psi1 = torch.from_numpy(p1np).to(dev)
    b = torch.empty((nrhs, p.nt, p.m), dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    prec = {"fp64": aao.AAO_PREC_FP64, "fp32": aao.AAO_PREC_FP32_IR, "f32x2": aao.AAO_PREC_F32X2}[
        WORKLOAD["precision"]]
    if varcoef:
        afun = p.meta["a"]
        s = aao.Solver(d, p.N, p.nt, p.tau, p.alpha, c2=W.grid_mean(afun, d, N), precision=prec,
                       nrhs_max=nrhs, variable_coefficient=True, graph=args.graph)
        s.set_coefficient(torch.from_numpy(np.concatenate(
            [fc.ravel() for fc in W.face_coefficients(afun, d, N)])).to(dev))
    else:
        s = aao.Solver(d, p.N, p.nt, p.tau, p.alpha, precision=prec, nrhs_max=nrhs, graph=args.graph)
    # kernel variants: measured on this GPU by the library's autotuner (untimed setup)
    variants = s.autotune() if args.autotune else None
    rtol, maxit = WORKLOAD["rtol"], WORKLOAD["maxit"]

    def step():
        s.build_rhs(f, psi0, psi1, b, stream=stream)
        st, info = s.solve(b, x, rtol=rtol, maxit=maxit, stream=stream)
        if st != aao.AAO_OK:
            raise RuntimeError(f"solve failed: {aao.aao_status_str(st)} {info}")
        return max(info, key=lambda i: i["iters"])

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize(dev)

    # per-kernel CUDA-event timing for the roofline: one profiled pass over the same
    # steps (kernel timing makes the library use its host-driven loop)
    aao.aao_profile_enable(s.h, True)
    for _ in range(max(1, min(args.steps, 5))):
        step()
    torch.cuda.synchronize(dev)
    prof = aao.aao_profile_read(s.h)
    aao.aao_profile_enable(s.h, False)

    clocks = ClockSampler(local)
    clocks.start()
    l0 = s.launches
    iters = []
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        iters.append(step()["iters"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ms = e0.elapsed_time(e1)
    launches = s.launches - l0
    clk = clocks.stop()
    ms_max = reduce_max(ms, world, dev)
    value = world * args.steps * nrhs / (ms_max / 1e3)
    it = float(np.mean(iters))
    relres = info["relres_true"]

    # ---- per-kernel roofline (live CUDA-event timing in the timed region) ----
    kern = {k: {"launches": v[0], "total_ms": round(v[1], 4), "avg_ms": v[1] / max(v[0], 1),
                "share": v[1] / max(sum(t for _, t in prof.values()), 1e-12)} for k, v in prof.items()}
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    hbm = measured_peaks().get("hbm_gbs", 6777.0)
    # FP32 time kernels read and write FP64 vectors except on the variable-coefficient
    # FP32 path, which keeps the whole P^{-1} in FP32 vectors
    vb32 = 4 if varcoef else 8

    def roof(cls):
        fl = algorithmic_flops(cls, d, p.N, p.nt, unknowns, varcoef)
        if cls.endswith("f32x2"):  # counted as the FP32 operations of the double-word algorithms
            fl *= DW_FP32_FLOPS_PER_FLOP
        fp64_cls = cls.endswith("f64") or cls.startswith("yt") or cls == "wx_res"
        by = algorithmic_bytes(cls, d, p.N, p.nt, unknowns, 8 if fp64_cls or cls.endswith("f32x2") else vb32)
        alu_peak = FP64_PEAK_TFLOPS if fp64_cls else FP32_PEAK_TFLOPS
        t = kern[cls]["avg_ms"] / 1e3
        # the binding roofline: whichever of the ALU and HBM times is longer
        if fl / (alu_peak * 1e12) >= by / (hbm * 1e9):
            return {"kernel": cls, "bound": "alu", "achieved": fl / t / 1e12, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": fl / t / 1e12 / alu_peak, "flops_per_launch": fl,
                    "bytes_per_launch": by,
                    "peak_note": ("FP64" if alu_peak == FP64_PEAK_TFLOPS else "FP32") +
                                 " CUDA-core peak from unit counts and clocks: 152 SMs x " +
                                 ("2 DFMA" if alu_peak == FP64_PEAK_TFLOPS else "128 FFMA") +
                                 "/clk x 2 flop x 2.07 GHz" +
                                 ("; achieved counts the FP32 flops of the double-word algorithms "
                                  "(%.1f per FP64-equivalent flop)" % DW_FP32_FLOPS_PER_FLOP
                                  if cls.endswith("f32x2") else "")}
        return {"kernel": cls, "bound": "hbm", "achieved": by / t / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": by / t / 1e9 / hbm, "flops_per_launch": fl, "bytes_per_launch": by,
                "peak_note": "measured copy bandwidth (of measured)"}

    roofline = roof(dom)
    if roofline["bound"] == "alu":
        # the unit-count peak stays the denominator; the measured FMA-loop rate is reported beside it
        meas = alu_peaks_measured()
        if meas:
            roofline["peak_measured_fma_loop"] = meas
            key = "fp64_tflops" if roofline["peak"] == FP64_PEAK_TFLOPS else "fp32_tflops"
            if meas.get(key):
                roofline["frac_of_measured_fma_loop"] = roofline["achieved"] / meas[key]
    var = None
    if variants:
        var = variants["time_variant"] if dom.startswith("time") else (
            variants["dst_variant"] if dom.startswith("dst") else None)
    roofline["traffic"] = traffic_record(dom, var)
    for k in kern:
        if algorithmic_flops(k, d, p.N, p.nt, unknowns, varcoef):
            r = roof(k)
            kern[k].update(bound=r["bound"], achieved=r["achieved"], unit=r["unit"], frac=r["frac"])
    # preconditioner application as a whole, against HBM (16 B per unknown in + out)
    prec_cls = [k for k in kern if k.startswith("dst") or k.startswith("time") or k == "cast"]
    applies = sum(v["launches"] for k, v in kern.items() if k.startswith("time"))
    prec_ms = sum(kern[k]["total_ms"] for k in prec_cls) / max(applies, 1)
    prec = {"ms_per_apply": prec_ms, "algorithmic_bytes": 16 * unknowns,
            "hbm_gbs": 16 * unknowns / (prec_ms / 1e3) / 1e9 if prec_ms else None}
    prec["frac_of_measured_hbm"] = prec["hbm_gbs"] / hbm if prec["hbm_gbs"] else None
    prec["frac_of_8tbs"] = prec["hbm_gbs"] / 8000.0 if prec["hbm_gbs"] else None

    # ---- end to end through the C ABI with host buffers ----
    if unknowns * 8 > 4e9:  # would pin more than 3 x 4 GB of host memory: not measured
        e2e = None
    else:
        fh = torch.from_numpy(fnp).pin_memory()
        p0h = torch.from_numpy(p0np).pin_memory()
        p1h = torch.from_numpy(p1np).pin_memory()
        uh = torch.empty((nrhs, p.nt, p.m), dtype=torch.float64).pin_memory()
        s.solve_host(fh, p0h, p1h, uh, rtol=rtol, maxit=maxit, stream=stream)  # staging warm-up
        e2e_steps = max(1, min(args.steps, 20))
        barrier(world)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            st, inf2 = s.solve_host(fh, p0h, p1h, uh, rtol=rtol, maxit=maxit, stream=stream)
            if st != aao.AAO_OK:
                raise RuntimeError(f"host solve failed {inf2}")
        torch.cuda.synchronize(dev)
        t_e2e = reduce_max(time.perf_counter() - t0, world, dev)
        barrier(world)
        e2e = {"value": world * e2e_steps * nrhs / t_e2e, "unit": "solves/s",
               "h2d_bytes_per_step": 8 * nrhs * (p.nt * p.m + 2 * p.m), "d2h_bytes_per_step": 8 * nrhs * p.nt * p.m,
               "steps": e2e_steps, "api": "aao_solve_host"}

    # ---- accuracy against the exact solution, the FP64 path and a cuFFT pipeline ----
    extra = {}
    if not varcoef and d < 3:
        xh = x[0].cpu().numpy()
        extra["error_vs_exact"] = error_vs_exact(xh, p)
        if WORKLOAD["precision"] != "fp64":
            with aao.Solver(d, p.N, p.nt, p.tau, p.alpha, nrhs_max=1, graph=args.graph) as s64:
                x64 = torch.empty_like(x[0])
                st64, info64 = s64.solve(b[0], x64, rtol=rtol, maxit=maxit, stream=stream)
                torch.cuda.synchronize(dev)
                extra["vs_fp64_gpu"] = {
                    "rel_diff_2norm": float(torch.linalg.norm(x[0] - x64) / torch.linalg.norm(x64)),
                    "fp64_iters": info64[0]["iters"], "fp64_relres_true": info64[0]["relres_true"],
                    "fp64_error_vs_exact": error_vs_exact(x64.cpu().numpy(), p)}
        elif d == 2 and rank == 0:
            extra["cufft_comparison"] = cufft_comparison(s, p, dev)

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline and args.workload == "2d255_fp64":
            pp, pc, A = oracle_problem()
            t_full, it_o = oracle_full_solve(pp, pc, A)
            cpu = {"value": 1.0 / t_full, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"one full oracle solve of the same workload (rhs + MINRES, {it_o} iterations, "
                             f"NumPy/BLAS on all host cores), {t_full:.2f} s; preconditioner setup excluded"}
            t_sp, it_sp, x_sp = scipy_fft_solve(p, rtol, maxit)
            xg = x[0].cpu().numpy()
            extra["cpu_fft_comparison"] = {
                "value": 1.0 / t_sp, "unit": "solves/s", "cores": os.cpu_count(), "iters": it_sp,
                "rel_diff_to_gpu": float(np.linalg.norm(x_sp - xg) / np.linalg.norm(xg)),
                "note": "the same solve restated with scipy.fft on all host cores (FFT-based DSTs and time "
                        "transforms, NumPy MINRES); a fair CPU-throughput reference beside the oracle"}
        out = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32+f64", "f32x2": "f32x2+f64"}[WORKLOAD["precision"]],
            "data": "synthetic", "config": workload_config(unknowns, args.workload),
            "iters_per_solve": it, "relres_true": relres,
            "unknown_iters_per_s": world * unknowns * it * args.steps / (ms_max / 1e3),
            "dtype_note": {"fp64": "f64 throughout",
                           "fp32": "f32/complex64 preconditioner; f64 operator, MINRES recurrences and refinement",
                           "f32x2": "preconditioner and DSTs in double-float (FP32 pairs, ~47 bits) on f64 "
                                    "vectors; f64 operator, MINRES recurrences and residuals"}[WORKLOAD["precision"]],
            "prec_apply": prec, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "kernels": kern, "kernel_variants": variants,
        }
        out.update(extra)
        if emit:
            print(json.dumps(out), flush=True)
    s.close()
    return out


def run_served(args, world, rank, local, emit=True):
    """Served stream: Poisson arrivals (mean --rate/s, default 200, seeded) of 1D/2D requests with mixed
    sizes, wave speeds and tolerances, admitted under a 120 GB HBM budget; replayed in
    real time; latency = completion - submission on the server's clock."""
    import numpy as np
    import torch

    import paper_2306_03574_gb300 as aao
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    count = args.requests
    rate = float(args.rate)
    sprec = aao.AAO_PREC_F32X2 if args.serve_precision == "f32x2" else aao.AAO_PREC_FP64
    reqs = W.served_requests(count=count, rate=rate, seed=5 + rank)
    # per-shape device data (source, initial values) shared by the requests of that shape;
    # wave speed, tolerance and the output buffer differ per request
    shapes = {}
    for r in reqs:
        key = (r["d"], r["N"], r["nt"])
        if key not in shapes:
            p = W.served_problem(r, alpha=1e-6)
            shapes[key] = dict(f=torch.from_numpy(p.f).to(dev), psi0=torch.from_numpy(p.psi0).to(dev),
                               psi1=torch.from_numpy(p.psi1).to(dev), m=p.m, free=[], tau=p.tau)
    srv = aao.aao_serve_create(int(120e9), args.slots)

    def out_buf(key):
        sh = shapes[key]
        if sh["free"]:
            return sh["free"].pop()
        return torch.empty((key[2], sh["m"]), dtype=torch.float64, device=dev)

    def submit(r, x):
        key = (r["d"], r["N"], r["nt"])
        sh = shapes[key]
        return aao.aao_serve_submit(srv, r["d"], r["N"], r["nt"], sh["tau"], 1e-6, r["c2"], r["tol"], 100,
                                    sh["f"], sh["psi0"], sh["psi1"], x, precision=sprec)

    # warm-up: one request per shape (handles, tables, captured graphs), untimed
    for key in shapes:
        r = next(q for q in reqs if (q["d"], q["N"], q["nt"]) == key)
        x = out_buf(key)
        st, _ = aao.aao_serve_wait(srv, submit(r, x), 300.0)
        shapes[key]["free"].append(x)
    torch.cuda.synchronize(dev)
    inflight = {}
    done = []
    sample = {}
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        while True:
            now = time.perf_counter() - t0
            for t in list(inflight):
                st, res = aao.aao_serve_poll(srv, t)
                if st == aao.AAO_EPENDING:
                    continue
                rr, x = inflight.pop(t)
                done.append((rr, st, res))
                key = (rr["d"], rr["N"], rr["nt"])
                if rr["id"] % 100 == 0 and rr["id"] not in sample:
                    sample[rr["id"]] = (rr, x.cpu().numpy())
                shapes[key]["free"].append(x)
            if now >= r["arrival"]:
                break
            time.sleep(min(2e-4, r["arrival"] - now))
        x = out_buf((r["d"], r["N"], r["nt"]))
        inflight[submit(r, x)] = (r, x)
    for t in list(inflight):
        st, res = aao.aao_serve_wait(srv, t, 600.0)
        rr, x = inflight.pop(t)
        done.append((rr, st, res))
        if rr["id"] % 100 == 0:
            sample[rr["id"]] = (rr, x.cpu().numpy())
    stats = aao.aao_serve_stats(srv)
    aao.aao_serve_destroy(srv)
    ok = [(rr, res) for rr, st, res in done if st == aao.AAO_OK]
    lat = np.array([res["t_done"] - res["t_submit"] for _, res in ok])
    t_first = min(res["t_submit"] for _, res in ok)
    t_last = max(res["t_done"] for _, res in ok)
    # each sampled result equals the same request solved alone (bit for bit); served
    # handles keep the standard tiles (their grouped launches use them), so the solo
    # handles are created with them too
    same = True
    small_env = os.environ.get("AAO_SMALL_TILES")
    os.environ["AAO_SMALL_TILES"] = "0"
    for rid, (rr, xs) in sample.items():
        key = (rr["d"], rr["N"], rr["nt"])
        sh = shapes[key]
        with aao.Solver(rr["d"], rr["N"], rr["nt"], sh["tau"], 1e-6, c2=rr["c2"], graph=True, precision=sprec) as s1:
            b = torch.empty((rr["nt"], sh["m"]), dtype=torch.float64, device=dev)
            s1.build_rhs(sh["f"], sh["psi0"], sh["psi1"], b)
            x1 = torch.empty_like(b)
            s1.solve(b, x1, rtol=rr["tol"], maxit=100)
            torch.cuda.synchronize(dev)
            same &= bool(np.array_equal(x1.cpu().numpy(), xs))
    if small_env is None:
        del os.environ["AAO_SMALL_TILES"]
    else:
        os.environ["AAO_SMALL_TILES"] = small_env
    unknowns = sum(rr["nt"] * rr["N"] ** rr["d"] for rr, _ in ok)
    line = {
        "metric": f"served solves/s with p50/p99 latency (Poisson {rate:g}/s, mixed 1D/2D, 120 GB budget)",
        "value": len(ok) / (t_last - t_first), "unit": "solves/s", "n_gpus": world,
        "steps": len(reqs), "warmup": len(shapes), "ms_per_step": 1e3 * (t_last - t_first) / max(len(ok), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.serve_precision == "fp64" else "f32x2+f64", "data": "synthetic",
        "config": {"workload": f"served_poisson{rate:g}_mixed_1d2d_{args.serve_precision}", "requests": len(reqs),
                   "slots": args.slots,
                   "budget_bytes": int(120e9), "shapes": len(shapes)},
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                       "mean": float(lat.mean() * 1e3), "max": float(lat.max() * 1e3)},
        "completed": len(ok), "failed": len(done) - len(ok), "offered_rate": rate,
        "unknowns_per_s": unknowns / (t_last - t_first), "iters_mean": float(np.mean([res["iters"] for _, res in ok])),
        "server": stats, "sample_equal_alone": same, "sample_size": len(sample),
    }
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def run_profile_case(args):
    """A small fixed case for ncu captures and variant timing: --reps applications of
    one step (--what) of one problem size through the C ABI, on seeded N(0,1) data.
    With --sweep, every time-kernel variant of the precision is timed with CUDA events
    (best of --reps after a warm-up) and one JSON line is printed."""
    import numpy as np
    import torch

    import paper_2306_03574_gb300 as aao

    if args.time_variant is not None:
        os.environ["AAO_TIME_VARIANT"] = f"{args.time_variant},{args.time_variant},{args.time_variant}"
    if args.dst_variant is not None:
        os.environ["AAO_DST_VARIANT"] = str(args.dst_variant)
    prec = {"fp64": aao.AAO_PREC_FP64, "fp32": aao.AAO_PREC_FP32_IR, "f32x2": aao.AAO_PREC_F32X2}[args.precision]
    d, N, nt = args.d, args.N, args.nt
    m = N ** d
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal((args.nrhs, nt, m))).cuda()
    y = torch.empty_like(x)

    def one(s):
        if args.what == "prec":
            s.apply_prec(x, y)
        elif args.what == "time":
            s.apply_time(x, y)
        elif args.what == "dst":
            s.apply_dst(x, y)
        elif args.what == "op":
            s.apply_op(x, y)
        else:
            s.apply_op(x, y)
            st, info = s.solve(y, x, rtol=1e-8, maxit=50)
            assert st == aao.AAO_OK, info

    if not args.sweep:
        # solves run host-driven (kernels of a graph with a WHILE node are not profiled)
        kw = dict(precision=prec, nrhs_max=args.nrhs, graph=args.what != "solve")
        if args.varcoef:  # Example 2's coefficient, mean-coefficient preconditioner
            import workloads as W
            afun = W.example2(N, nt).meta["a"]
            kw.update(variable_coefficient=True, c2=W.grid_mean(afun, d, N))
        with aao.Solver(d, N, nt, 1.0 / nt, args.pc_alpha, **kw) as s:
            if args.varcoef:
                s.set_coefficient(torch.from_numpy(np.concatenate(
                    [fc.ravel() for fc in W.face_coefficients(afun, d, N)])).cuda())
            for _ in range(args.reps):
                one(s)
            torch.cuda.synchronize()
        print("ok")
        return 0
    nvar = {"fp64": 8, "fp32": 34, "f32x2": 15}[args.precision]
    times = {}
    # --what dst sweeps the DST variants (8: the small-problem tile), else the time
    # kernel's (30: the small-problem tile)
    sweep = range(9) if args.what == "dst" else sorted(set(range(nvar)) | {30})
    for v in sweep:
        if args.what == "dst":
            os.environ["AAO_DST_VARIANT"] = str(v)
        else:
            os.environ["AAO_TIME_VARIANT"] = f"{v},{v},{v}"
        with aao.Solver(d, N, nt, 1.0 / nt, args.pc_alpha, precision=prec, nrhs_max=args.nrhs) as s:
            one(s)
            torch.cuda.synchronize()
            best = 1e30
            for _ in range(max(args.reps, 3)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                one(s)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            times[v] = best
    print(json.dumps({"profile_case": {"d": d, "N": N, "nt": nt, "nrhs": args.nrhs, "precision": args.precision,
                                       "what": args.what}, "variant_ms": times,
                      "wait_timeouts": aao.aao_wait_timeouts()}), flush=True)
    return 0


def _summary(line):
    """The figures of one workload's line that the default line carries."""
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "iters_per_solve", "relres_true",
            "unknown_iters_per_s", "roofline", "clocks", "e2e", "error_vs_exact", "vs_fp64_gpu", "gpu_launches",
            "latency_ms", "completed", "failed", "offered_rate", "sample_equal_alone", "sample_size",
            "kernel_variants")
    out = {k: line[k] for k in keep if k in line}
    out["config"] = line.get("config")
    if "server" in line:
        srv = line["server"]
        out["server"] = {k: srv[k] for k in ("rounds", "round_problems", "grouped_launches", "handles_created",
                                             "evictions", "peak_pool_bytes") if k in srv}
    return out


def run_extra_workloads(args, world, rank, local):
    """The other configurations of the benchmark, each measured as its own workload
    (own warm-up, CUDA-event timing, clocks and roofline): the 1D 63 x 64 latency case,
    the 2D 511^2 x 512 mixed-precision case and a served Poisson stream."""
    import copy
    res = {}
    saved = dict(WORKLOAD), WORKLOAD_NAME[0]
    for name, steps in (("1d63_fp64", 50), ("2d511_mixed", 10)):
        a = copy.copy(args)
        a.workload, a.steps, a.warmup, a.no_cpu_baseline = name, steps, 3, True
        WORKLOAD.clear()
        WORKLOAD.update(WORKLOADS[name])
        WORKLOAD_NAME[0] = name
        try:
            res[name] = _summary(run_gpu(a, world, rank, local, emit=False))
        except Exception as e:  # report, keep the default line
            res[name] = {"error": repr(e)[:300]}
    WORKLOAD.clear()
    WORKLOAD.update(saved[0])
    WORKLOAD_NAME[0] = saved[1]
    a = copy.copy(args)
    a.workload, a.requests = "served", args.served_requests
    try:
        res["served"] = _summary(run_served(a, world, rank, local, emit=False))
    except Exception as e:
        res["served"] = {"error": repr(e)[:300]}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["served"], default="2d255_fp64")
    ap.add_argument("--requests", type=int, default=2000, help="served workload: number of requests")
    ap.add_argument("--served-requests", type=int, default=400,
                    help="requests of the served stream reported under 'workloads' by the default run")
    ap.add_argument("--slots", type=int, default=8, help="served workload: concurrent solves")
    ap.add_argument("--rate", type=float, default=200.0, help="served workload: mean Poisson arrival rate (1/s)")
    ap.add_argument("--serve-precision", choices=["fp64", "f32x2"], default="fp64",
                    help="served workload: precision mode of every request")
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--graph", type=int, default=1,
                    help="1: solve loop captured in a CUDA graph (device-side while loop); 0: host-driven")
    ap.add_argument("--extra-workloads", type=int, default=1,
                    help="default workload at N=1: also measure the 1D latency, 2D 511^2 x 512 mixed-precision "
                         "and served-stream workloads and report them under 'workloads'")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: pick the time/DST kernel variants by measurement before warm-up; 0: defaults")
    pc = ap.add_argument_group("--profile-case: one small fixed case (ncu captures, variant timing)")
    pc.add_argument("--profile-case", action="store_true")
    pc.add_argument("--what", choices=["prec", "time", "dst", "op", "solve"], default="prec")
    pc.add_argument("--d", type=int, default=2)
    pc.add_argument("--N", type=int, default=255)
    pc.add_argument("--nt", type=int, default=256)
    pc.add_argument("--nrhs", type=int, default=1)
    pc.add_argument("--precision", choices=["fp64", "fp32", "f32x2"], default="fp64")
    pc.add_argument("--pc-alpha", type=float, default=1e-6)
    pc.add_argument("--reps", type=int, default=1)
    pc.add_argument("--time-variant", type=int, default=None)
    pc.add_argument("--dst-variant", type=int, default=None)
    pc.add_argument("--sweep", action="store_true", help="time every time-kernel variant")
    pc.add_argument("--varcoef", action="store_true", help="Example 2's variable coefficient (2D)")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.workload != "served":
        WORKLOAD.clear()
        WORKLOAD.update(WORKLOADS[args.workload])
        WORKLOAD_NAME[0] = args.workload
        if args.alpha is not None:
            WORKLOAD["alpha"] = args.alpha
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        world, rank, local = dist_setup(args.gpus, "gloo")
        rc = run_reference(args, world, rank)
    elif args.workload == "served":
        world, rank, local = dist_setup(args.gpus, "nccl")
        run_served(args, world, rank, local)
        rc = 0
    else:
        world, rank, local = dist_setup(args.gpus, "nccl")
        if args.workload == "2d255_fp64" and args.extra_workloads and world == 1:
            out = run_gpu(args, world, rank, local, emit=False)
            out["workloads"] = run_extra_workloads(args, world, rank, local)
            print(json.dumps(out), flush=True)
        else:
            run_gpu(args, world, rank, local)
        rc = 0
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
