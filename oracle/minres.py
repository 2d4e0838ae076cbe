"""Textbook preconditioned MINRES (oracle; test infrastructure only).

The paper runs MINRES with the SPD preconditioner P_alpha on Y T u = Y f
(eq. (precsys)), zero initial guess (Section 3), and analyses it through the
bound of Lemma minrescvglm (Elman-Silvester-Wathen, Theorem 6.13).  This is
the standard Lanczos + Givens form of preconditioned MINRES: with P = L L^T
it is MINRES on L^{-1} A L^{-T}, rewritten so that only P^{-1} is applied.

Stopping rule (a reading: Section 3 states "relative residual" 1e-6): stop at
the first iteration j whose TRUE relative residual ||b - A x_j||_2 / ||b||_2 is
<= rtol (recomputed explicitly each iteration), or at maxit.  The recurrence
estimate |eta_j| / gamma_1 = ||r_j||_{P^{-1}} / ||r_0||_{P^{-1}} is returned too.
"""
from __future__ import annotations

import numpy as np


def minres(apply_A, apply_Minv, b: np.ndarray, x0=None, rtol: float = 1e-8,
           maxit: int = 200, true_residual: bool = True):
    """Returns (x, info) with info = dict(iters, relres_true, relres_est,
    history_est, history_true, breakdown)."""
    dot = lambda a, c: float(np.vdot(a.ravel(), c.ravel()).real)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    nb = np.linalg.norm(b)
    v_prev = np.zeros_like(b)
    v = b - apply_A(x) if x0 is not None else b.copy()
    z = apply_Minv(v)
    gam2 = dot(z, v)
    info = dict(iters=0, relres_true=np.linalg.norm(v) / nb if nb > 0 else 0.0,
                relres_est=1.0, history_est=[], history_true=[], breakdown=False)
    if gam2 <= 0.0 or nb == 0.0:
        info["breakdown"] = gam2 < 0.0
        return x, info
    gam = np.sqrt(gam2)
    gam_prev = 1.0
    gam1 = gam
    eta = gam
    c_prev, c = 1.0, 1.0
    s_prev, s = 0.0, 0.0
    w_prev = np.zeros_like(b)
    w = np.zeros_like(b)
    for j in range(1, maxit + 1):
        z = z / gam                                    # normalised z_j
        Az = apply_A(z)
        delta = dot(Az, z)
        v_next = Az - (delta / gam) * v - (gam / gam_prev) * v_prev
        z_next = apply_Minv(v_next)
        g2 = dot(z_next, v_next)
        if g2 < 0.0:
            info["breakdown"] = True
            break
        gam_next = np.sqrt(g2)
        # Givens rotation eliminating gam_next from the tridiagonal column
        a0 = c * delta - c_prev * s * gam
        a1 = np.sqrt(a0 * a0 + gam_next * gam_next)
        a2 = s * delta + c_prev * c * gam
        a3 = s_prev * gam
        c_next = a0 / a1
        s_next = gam_next / a1
        w_next = (z - a3 * w_prev - a2 * w) / a1
        x = x + c_next * eta * w_next
        eta = -s_next * eta
        # shift
        v_prev, v = v, v_next
        z = z_next
        gam_prev, gam = gam, gam_next
        c_prev, c = c, c_next
        s_prev, s = s, s_next
        w_prev, w = w, w_next
        info["iters"] = j
        info["relres_est"] = abs(eta) / gam1
        info["history_est"].append(info["relres_est"])
        if true_residual:
            rt = np.linalg.norm(b - apply_A(x)) / nb
            info["relres_true"] = rt
            info["history_true"].append(rt)
            if rt <= rtol:
                break
        elif info["relres_est"] <= rtol:
            break
        if gam_next == 0.0:
            break
    if not true_residual:
        info["relres_true"] = np.linalg.norm(b - apply_A(x)) / nb
    return x, info
