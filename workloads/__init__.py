"""Seeded synthetic inputs for the all-at-once wave solver.

This module is shared by the CPU oracle and by the GPU path, so it holds no
arithmetic of the method itself: it only evaluates the model problem's data
(grids, initial values psi0/psi1, source samples f^(k), manufactured exact
solutions) and draws seeded random numbers.  Building the all-at-once
right-hand side, applying the operator or the preconditioner is done
separately by each side.

Conventions (paper, Section 1, eq. (1.1) and the scheme below it):
  * Omega = (0,1)^d, homogeneous Dirichlet boundary, N interior points per axis,
    h = 1/(N+1), grid points x_i = i*h, i = 1..N.
  * Spatial points are ordered lexicographically with x fastest, so a
    spatial field has numpy shape (N,)*d indexed [.., iy, ix] (C order).
  * tau = T/n; the unknowns are u^(1..n) at t = k*tau, k = 1..n; the source is
    sampled as f^(k) = f(G_h, k*tau) for k = 0..n-1.
  * An all-at-once vector is time-major: shape (n, m) with m = N**d.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

__all__ = [
    "WaveProblem", "grid_axes", "make_rng", "random_field",
    "config_1d", "config_2d", "config_2d_large", "config_3d_batched",
    "example1", "example2", "served_requests", "face_coefficients", "grid_mean",
]


def make_rng(seed: int) -> np.random.Generator:
    """PCG64 generator; every input in this project is drawn from one."""
    return np.random.Generator(np.random.PCG64(seed))


def grid_axes(d: int, N: int):
    """Meshgrid coordinate arrays (x, y, z...) of the interior points.

    Returned arrays have shape (N,)*d indexed [.., iy, ix]; element 0 is x.
    """
    h = 1.0 / (N + 1)
    g = np.arange(1, N + 1, dtype=np.float64) * h
    mesh = np.meshgrid(*([g] * d), indexing="ij")  # mesh[a] varies along array axis a
    # array axis 0 is the slowest (z or y), the last axis is x
    return tuple(mesh[d - 1 - a] for a in range(d))


@dataclass
class WaveProblem:
    """One synthetic instance of u_tt = c^2 Lap u + f with its data sampled on the grid.

    f has shape (n, m): f[k] = f^(k) at t = k*tau (k = 0..n-1), flattened spatially.
    psi0, psi1 have shape (m,).  exact(t) returns u(G_h, t) flattened, or None.
    """
    d: int
    N: int
    nt: int
    T: float
    c2: float
    alpha: float
    psi0: np.ndarray
    psi1: np.ndarray
    f: np.ndarray
    exact: Optional[Callable[[float], np.ndarray]] = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.N ** self.d

    @property
    def h(self) -> float:
        return 1.0 / (self.N + 1)

    @property
    def tau(self) -> float:
        return self.T / self.nt

    def exact_levels(self) -> Optional[np.ndarray]:
        """Exact solution at t = k*tau, k = 1..n, shape (n, m)."""
        if self.exact is None:
            return None
        return np.stack([self.exact(k * self.tau) for k in range(1, self.nt + 1)])


def random_field(shape, seed: int, dist: str = "normal") -> np.ndarray:
    """Seeded random FP64 array (normal(0,1) or uniform[-1,1])."""
    rng = make_rng(seed)
    if dist == "normal":
        return rng.standard_normal(shape)
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=shape)
    raise ValueError(dist)


def config_1d(N: int = 63, nt: int = 64, alpha: float = 1e-6, seed: int = 1,
              noise: float = 1e-3, c2: float = 1.0) -> WaveProblem:
    """1D wave on [0,1]x[0,1]: manufactured u = sin(pi x) cos(pi t) (so f = 0),
    plus seeded N(0, noise^2) source noise on every grid point and time level."""
    (x,) = grid_axes(1, N)
    c = np.sqrt(c2)
    psi0 = np.sin(np.pi * x).ravel()
    psi1 = np.zeros_like(psi0)
    f = noise * make_rng(seed).standard_normal((nt, N))
    exact = lambda t: (np.sin(np.pi * x) * np.cos(c * np.pi * t)).ravel()
    return WaveProblem(1, N, nt, 1.0, c2, alpha, psi0, psi1, f, exact,
                       name=f"1d_N{N}_nt{nt}")


def config_2d(N: int = 255, nt: int = 256, alpha: float = 1e-6, seed: int = 2,
              noise: float = 1e-3, c2: float = 1.0) -> WaveProblem:
    """2D wave on [0,1]^2: manufactured u = sin(pi x) sin(pi y) cos(sqrt(2) pi t)
    (so f = 0), plus seeded noise*U[-1,1] source noise."""
    x, y = grid_axes(2, N)
    c = np.sqrt(c2)
    base = np.sin(np.pi * x) * np.sin(np.pi * y)
    psi0 = base.ravel().copy()
    psi1 = np.zeros_like(psi0)
    f = noise * make_rng(seed).uniform(-1.0, 1.0, size=(nt, N * N))
    exact = lambda t: (base * np.cos(c * np.sqrt(2.0) * np.pi * t)).ravel()
    return WaveProblem(2, N, nt, 1.0, c2, alpha, psi0, psi1, f, exact,
                       name=f"2d_N{N}_nt{nt}")


def config_2d_large(seed: int = 3, alpha: float = 1e-6) -> WaveProblem:
    """2D wave as config_2d on a 511x511 interior grid with 512 time levels."""
    p = config_2d(N=511, nt=512, alpha=alpha, seed=seed)
    p.name = "2d_N511_nt512"
    return p


def config_3d_batched(N: int = 127, nt: int = 128, nrhs: int = 8, seed: int = 4,
                      alpha: float = 1e-6):
    """3D wave, zero initial data, nrhs seeded N(0,1) sources.

    Returns (problem_template, f_batch) with f_batch shape (nrhs, nt, N^3).
    The template's f is the first right-hand side.
    """
    m = N ** 3
    rng = make_rng(seed)
    fb = rng.standard_normal((nrhs, nt, m))
    z = np.zeros(m)
    p = WaveProblem(3, N, nt, 1.0, 1.0, alpha, z, z.copy(), fb[0], None,
                    name=f"3d_N{N}_nt{nt}_x{nrhs}")
    return p, fb


def example1(N: int, nt: int, alpha: float = 1e-6) -> WaveProblem:
    """The paper's Example 1 (Section 3): d = 2, T = 1,
    psi0 = -psi1 = x1(x1-1)x2(x2-1), u = exp(-t) x1(x1-1)x2(x2-1)."""
    x, y = grid_axes(2, N)
    p = x * (x - 1.0) * y * (y - 1.0)
    q = x * (x - 1.0) + y * (y - 1.0)
    psi0 = p.ravel().copy()
    psi1 = -psi0
    tau = 1.0 / nt
    f = np.stack([(np.exp(-k * tau) * (p - 2.0 * q)).ravel() for k in range(nt)])
    exact = lambda t: (np.exp(-t) * p).ravel()
    return WaveProblem(2, N, nt, 1.0, 1.0, alpha, psi0, psi1, f, exact,
                       name=f"example1_N{N}_nt{nt}")


def example2(N: int, nt: int, alpha: float = 1e-6) -> WaveProblem:
    """The paper's Example 2 (Section 3, variable coefficient): d = 2, T = 1,
    a = (30 + sin^2 x1)(30 + sin^2 x2), psi0 = psi1 = x1(1-x1)x2(1-x2),
    u = exp(t) x1(1-x1)x2(1-x2).  meta['a'] holds the coefficient function."""
    x, y = grid_axes(2, N)
    A = 30.0 + np.sin(x) ** 2
    B = 30.0 + np.sin(y) ** 2
    q = x * (1.0 - x) * y * (1.0 - y)
    psi0 = q.ravel().copy()
    psi1 = psi0.copy()
    tau = 1.0 / nt
    src = (q - np.sin(2 * x) * B * (1 - 2 * x) * y * (1 - y)
           - np.sin(2 * y) * A * (1 - 2 * y) * x * (1 - x)
           + 2 * A * B * (x * (1 - x) + y * (1 - y)))
    f = np.stack([(np.exp(k * tau) * src).ravel() for k in range(nt)])
    exact = lambda t: (np.exp(t) * q).ravel()
    afun = lambda X, Y: (30.0 + np.sin(X) ** 2) * (30.0 + np.sin(Y) ** 2)
    return WaveProblem(2, N, nt, 1.0, 1.0, alpha, psi0, psi1, f, exact,
                       name=f"example2_N{N}_nt{nt}", meta={"a": afun})


def face_coefficients(afun, d: int, N: int):
    """A coefficient function sampled on the cell faces: for axis ax (0 = x) an array of
    shape (N,)*d with axis ax extended to N+1 faces, face f at coordinate (f + 1/2) h
    along ax (f = 0..N) and grid-point coordinates along the other axes (array axis 0
    is the slowest coordinate).  afun takes coordinate arrays (x, y, ...)."""
    h = 1.0 / (N + 1)
    g = np.arange(1, N + 1) * h
    fg = (np.arange(N + 1) + 0.5) * h
    out = []
    for ax in range(d):
        axes = [fg if (d - 1 - a) == ax else g for a in range(d)]
        mesh = np.meshgrid(*axes, indexing="ij")
        out.append(afun(*[mesh[d - 1 - c] for c in range(d)]))
    return out


def grid_mean(afun, d: int, N: int) -> float:
    """Mean of a coefficient function over the grid points."""
    return float(np.mean(afun(*grid_axes(d, N))))


def served_requests(count: int = 2000, rate: float = 200.0, seed: int = 5,
                    max_2d_N: int = 255, max_1d_nt: int = 1024, max_2d_nt: int = 512):
    """Seeded request stream for the serving workload.

    Poisson arrivals (exponential gaps, mean 1/rate s); each request is 1D or 2D
    with probability 1/2; 1D N in {63,127,255,511}, nt in {64..max_1d_nt};
    2D N in {63,127,..,max_2d_N}, nt in {64..max_2d_nt} (powers of two);
    c ~ U[0.5, 2]; tol in {1e-6, 1e-8}.  Returns a list of dicts.
    """
    rng = make_rng(seed)
    t = 0.0
    out = []
    nts1 = [v for v in (64, 128, 256, 512, 1024) if v <= max_1d_nt]
    nts2 = [v for v in (64, 128, 256, 512) if v <= max_2d_nt]
    Ns2 = [v for v in (63, 127, 255) if v <= max_2d_N]
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        d = 1 if rng.random() < 0.5 else 2
        if d == 1:
            N = int(rng.choice([63, 127, 255, 511]))
            nt = int(rng.choice(nts1))
        else:
            N = int(rng.choice(Ns2))
            nt = int(rng.choice(nts2))
        c = float(rng.uniform(0.5, 2.0))
        tol = float(rng.choice([1e-6, 1e-8]))
        out.append(dict(id=i, arrival=t, d=d, N=N, nt=nt, c2=c * c, tol=tol,
                        seed=1000 + i))
    return out


def served_problem(req: dict, alpha: float = 1e-6) -> WaveProblem:
    """Problem data of one served request (same manufactured data as the 1D/2D
    configs with the requested wave speed)."""
    if req["d"] == 1:
        return config_1d(N=req["N"], nt=req["nt"], alpha=alpha, seed=req["seed"], c2=req["c2"])
    return config_2d(N=req["N"], nt=req["nt"], alpha=alpha, seed=req["seed"], c2=req["c2"])
