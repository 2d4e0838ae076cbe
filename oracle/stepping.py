"""Sequential time stepping of the implicit leap-frog scheme (oracle; test infrastructure only).

Block forward substitution with the lower-triangular T of eq. (main_matrix):
  L u_1 = f_1;  L u_2 = f_2 + 2 u_1;  L u_k = f_k + 2 u_{k-1} - L u_{k-2}  (k >= 3),
i.e. u_k = L^{-1}(f_k + 2 u_{k-1}) - u_{k-2}.  L is factorised by a sparse LU
(a library routine, independent of the DST diagonalisation).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .system import L_matrix, rhs_f


def sequential_solve(prob, f_all: np.ndarray = None, L=None) -> np.ndarray:
    """u^(1..n) of the scheme, shape (n, m); f_all defaults to eq. (main_matrix)'s f;
    L (sparse) defaults to I - (c^2 tau^2/2) Delta_h (pass L_a for the variable coefficient)."""
    L = (L_matrix(prob.d, prob.N, prob.tau, prob.c2) if L is None else L).tocsc()
    lu = spla.splu(L)
    f = rhs_f(prob) if f_all is None else f_all
    n = f.shape[0]
    u = np.zeros_like(f)
    for k in range(n):
        r = f[k].copy()
        if k >= 1:
            r = r + 2.0 * u[k - 1]
        u[k] = lu.solve(r)
        if k >= 2:
            u[k] -= u[k - 2]
    return u
