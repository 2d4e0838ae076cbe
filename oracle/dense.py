"""Dense tiny-size forms of the preconditioner (oracle; test infrastructure only).

  * C_alpha^{1/2} by the Schur method (scipy.linalg.sqrtm) and by an
    eigendecomposition with the principal branch (eq. (calphasqrtdiagform));
  * P_alpha = (C_alpha^{1/2})^T C_alpha^{1/2} (def. (matrix_P)) and P_alpha^{-1} y
    by a Cholesky solve;
  * the ideal preconditioner (T^{1/2})^T T^{1/2} (Proposition ideal_P);
  * the alpha = 1 ABC case |C_1| = sqrt(C_1^T C_1) (Remark p1badpermformremark).
Sizes are limited to m*n of a few thousand.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def sqrtm_schur(A: np.ndarray) -> np.ndarray:
    """Principal square root by the (complex) Schur method."""
    r = sla.sqrtm(A)
    return r[0] if isinstance(r, tuple) else r


def sqrtm_eig(A: np.ndarray) -> np.ndarray:
    """Principal square root through A = X diag(mu) X^{-1}: X diag(sqrt(mu)) X^{-1}."""
    mu, X = np.linalg.eig(A)
    return (X * np.sqrt(mu.astype(np.complex128))[None, :]) @ np.linalg.inv(X)


def P_alpha_dense(C: np.ndarray, method: str = "schur") -> np.ndarray:
    """P_alpha = (C^{1/2})^T C^{1/2} (real part; the imaginary part is round-off)."""
    R = sqrtm_schur(C) if method == "schur" else sqrtm_eig(C)
    P = R.T @ R
    return P


def prec_solve_dense(P: np.ndarray, y: np.ndarray) -> np.ndarray:
    """P^{-1} y by a Cholesky factorisation of the SPD matrix P."""
    c = sla.cho_factor(P.real)
    return sla.cho_solve(c, y)


def ideal_preconditioner(T: np.ndarray) -> np.ndarray:
    """(T^{1/2})^T T^{1/2} with T^{1/2} the principal square root."""
    R = sqrtm_schur(T).real
    return R.T @ R


def abs_sym(H: np.ndarray) -> np.ndarray:
    """|H| = sqrt(H^* H) for a real matrix, by the SVD (polar decomposition)."""
    U, s, Vt = np.linalg.svd(H)
    return (Vt.T * s[None, :]) @ Vt
