"""Pins for the variable-coefficient oracle (Section 3, eq. (var coeff wave),
eq. (tssystemvarwaveeq), the mean-coefficient preconditioner eq. (mean-coefftsmat),
Example 2 and Table 3)."""
import numpy as np
import pytest

import workloads as W
from oracle import fast as F
from oracle import minres as M
from oracle import stepping as ST
from oracle import system as S


def _afun(x, y):
    return (30.0 + np.sin(x) ** 2) * (30.0 + np.sin(y) ** 2)


@pytest.mark.parametrize("d,N", [(1, 7), (2, 5), (3, 3)])
def test_constant_coefficient_reduces_to_L(d, N):
    """a = c^2 everywhere: L_a = I - (c^2 tau^2/2) Delta_h."""
    tau = 0.3
    faces = S.face_coefficients(lambda *c: np.full_like(c[0], 2.5), d, N)
    v = np.random.default_rng(1).standard_normal((4, N ** d))
    assert np.abs(S.apply_La_stencil(v, faces, d, N, tau) - S.apply_L_stencil(v, d, N, tau, 2.5)).max() < 1e-12


@pytest.mark.parametrize("d,N", [(1, 9), (2, 6), (3, 4)])
def test_stencil_equals_independent_assembly(d, N):
    """Stencil == D^T diag(a) D assembly; L_a symmetric positive definite."""
    tau = 0.05
    af = (lambda x: 1 + x ** 2) if d == 1 else (_afun if d == 2 else (lambda x, y, z: 1 + x * y + z))
    faces = S.face_coefficients(af, d, N)
    La = S.La_matrix(faces, d, N, tau)
    v = np.random.default_rng(2).standard_normal(N ** d)
    assert np.abs(S.apply_La_stencil(v, faces, d, N, tau) - La @ v).max() < 1e-12 * np.abs(La @ v).max()
    Ld = La.toarray()
    assert np.abs(Ld - Ld.T).max() == 0.0
    assert np.linalg.eigvalsh(Ld).min() > 1.0


def test_second_order_consistency():
    """(Delta_{a,h} u)(x) -> div(a grad u)(x) at O(h^2) for Example 2's spatial profile."""
    errs = []
    for N in (15, 31, 63):
        x, y = W.grid_axes(2, N)
        q = (x * (1 - x) * y * (1 - y)).ravel()
        faces = S.face_coefficients(_afun, 2, N)
        tau = 1.0
        lap = -(S.apply_La_stencil(q, faces, 2, N, tau) - q) * 2.0 / (tau * tau)
        A = 30 + np.sin(x) ** 2
        B = 30 + np.sin(y) ** 2
        exact = (np.sin(2 * x) * B * (1 - 2 * x) * y * (1 - y) + np.sin(2 * y) * A * (1 - 2 * y) * x * (1 - x)
                 - 2 * A * B * (x * (1 - x) + y * (1 - y))).ravel()
        errs.append(np.abs(lap - exact).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_all_at_once_equals_sequential_variable():
    p = W.example2(7, 16)
    faces = S.face_coefficients(p.meta["a"], 2, 7)
    b = S.rhs_b_var(p, faces)
    La = S.La_matrix(faces, 2, 7, p.tau)
    u_seq = ST.sequential_solve(p, f_all=b[::-1].copy(), L=La)
    x, y = W.grid_axes(2, 7)
    pc = F.ABACPreconditioner(2, 7, 16, p.tau, 1e-6, c2=float(np.mean(p.meta["a"](x, y))))
    u, info = M.minres(lambda v: S.apply_YT_var(v, faces, 2, 7, p.tau), pc.apply, b, rtol=1e-14, maxit=200)
    assert np.abs(u - u_seq).max() < 1e-11 * np.abs(u_seq).max()


@pytest.mark.parametrize("lt,lh", [(4, 4), (4, 5), (5, 4), (5, 5), (6, 4), (7, 4)])
def test_table3_iterations(lt, lh):
    """Table 3, MINRES-P_alpha with the mean-coefficient preconditioner (alpha = 1e-6,
    tol 1e-6): 8-10 iterations, flat in tau and h (the paper prints 8 for these tau
    except 10 at tau = 2^-7)."""
    nt, N = 2 ** lt, 2 ** lh - 1
    p = W.example2(N, nt)
    faces = S.face_coefficients(p.meta["a"], 2, N)
    x, y = W.grid_axes(2, N)
    pc = F.ABACPreconditioner(2, N, nt, p.tau, 1e-6, c2=float(np.mean(p.meta["a"](x, y))))
    _, info = M.minres(lambda v: S.apply_YT_var(v, faces, 2, N, p.tau), pc.apply, S.rhs_b_var(p, faces),
                       rtol=1e-6, maxit=60)
    assert 8 <= info["iters"] <= 10
