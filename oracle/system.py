"""All-at-once system of the implicit leap-frog wave scheme (oracle; test infrastructure only).

Paper references:
  * scheme: Section 1, the leap-frog difference equation for k = 1..n-1
  * all-at-once matrix T and right-hand side f: eq. (main_matrix)
  * L = I_m - (tau^2/2) Delta_h (with wave speed: c^2 tau^2 / 2)
  * symmetrisation Y = Y_n (x) I_m: eqs. (symmetricform), (main_system)
  * block alpha-circulant C_alpha: def. (matrix_C_alpha); split (C_decom)
  * error E_{tau,h}: Section 3
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def laplacian_1d(N: int) -> sp.csr_matrix:
    """Second-order 3-point Dirichlet Laplacian on N interior points, h = 1/(N+1)."""
    h = 1.0 / (N + 1)
    e = np.ones(N)
    return sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], format="csr") / (h * h)


def laplacian(d: int, N: int) -> sp.csr_matrix:
    """(2d+1)-point Dirichlet Laplacian Delta_h on the uniform grid, lexicographic
    order with x fastest: a Kronecker sum of 1D Laplacians."""
    T1 = laplacian_1d(N)
    I = sp.identity(N, format="csr")
    out = None
    for a in range(d):
        # axis a (0 = x) is the a-th fastest index
        mats = [I] * d
        mats[d - 1 - a] = T1
        k = mats[0]
        for M in mats[1:]:
            k = sp.kron(k, M, format="csr")
        out = k if out is None else out + k
    return out.tocsr()


def L_matrix(d: int, N: int, tau: float, c2: float = 1.0) -> sp.csr_matrix:
    """L = I_m - (c^2 tau^2 / 2) Delta_h (below eq. (main_matrix); c^2 = 1 in the paper)."""
    m = N ** d
    return (sp.identity(m, format="csr") - 0.5 * c2 * tau * tau * laplacian(d, N)).tocsr()


def T_matrix(L: sp.spmatrix, n: int) -> sp.csr_matrix:
    """Block lower-triangular Toeplitz all-at-once matrix of eq. (main_matrix):
    block row 1 = [L], row 2 = [-2I, L], row k >= 3 = [.., L, -2I, L]."""
    m = L.shape[0]
    I = sp.identity(m, format="csr")
    blocks = [[None] * n for _ in range(n)]
    for i in range(n):
        blocks[i][i] = L
        if i >= 1:
            blocks[i][i - 1] = -2.0 * I
        if i >= 2:
            blocks[i][i - 2] = L
    return sp.bmat(blocks, format="csr")


def Y_matrix(n: int, m: int) -> sp.csr_matrix:
    """Y = Y_n (x) I_m with Y_n the n x n anti-identity (eq. (main_system))."""
    Yn = sp.csr_matrix(np.fliplr(np.eye(n)))
    return sp.kron(Yn, sp.identity(m), format="csr")


def B_alpha(n: int, alpha: float):
    """B_1^(alpha), B_2^(alpha) of eq. (C_decom), written out entry by entry."""
    B1 = np.zeros((n, n))
    B2 = np.zeros((n, n))
    for i in range(n):
        B1[i, i] = 1.0
        if i >= 2:
            B1[i, i - 2] = 1.0
        if i >= 1:
            B2[i, i - 1] = 1.0
    B1[0, n - 2] += alpha   # (1, n-1) in 1-based indexing
    B1[1, n - 1] += alpha   # (2, n)
    B2[0, n - 1] += alpha   # (1, n)
    return B1, B2


def C_alpha_matrix(L: sp.spmatrix, n: int, alpha: float) -> sp.csr_matrix:
    """C_alpha of def. (matrix_C_alpha): T plus the wrap-around blocks alpha*L,
    -2*alpha*I in block row 1 (block columns n-1, n) and alpha*L in block row 2
    (block column n).  Blocks are accumulated, so n = 2 also follows the pattern."""
    m = L.shape[0]
    I = sp.identity(m, format="csr")
    blocks = {}
    def add(bi, bj, M):
        blocks[(bi, bj)] = blocks[(bi, bj)] + M if (bi, bj) in blocks else M
    for i in range(n):
        add(i, i, L)
        if i >= 1:
            add(i, i - 1, -2.0 * I)
        if i >= 2:
            add(i, i - 2, L)
    add(0, n - 2, alpha * L)
    add(0, n - 1, -2.0 * alpha * I)
    add(1, n - 1, alpha * L)
    grid = [[blocks.get((i, j)) for j in range(n)] for i in range(n)]
    return sp.bmat(grid, format="csr")


def C_alpha_from_split(L: sp.spmatrix, n: int, alpha: float) -> sp.csr_matrix:
    """C_alpha = B_1 (x) L + B_2 (x) (-2 I_m), eq. (C_decom)."""
    B1, B2 = B_alpha(n, alpha)
    m = L.shape[0]
    return (sp.kron(sp.csr_matrix(B1), L) + sp.kron(sp.csr_matrix(B2), -2.0 * sp.identity(m))).tocsr()


def rhs_f(prob) -> np.ndarray:
    """Right-hand side f of eq. (main_matrix), shape (n, m):
    tau^2 [ f^0/2 + psi1/tau + psi0/tau^2 ; f^1 - L psi0/tau^2 ; f^2 ; ... ; f^(n-1) ].
    (The first block follows the paper literally.)"""
    tau = prob.tau
    L = L_matrix(prob.d, prob.N, tau, prob.c2)
    F = np.array(prob.f, dtype=np.float64, copy=True)
    out = tau * tau * F
    out[0] = tau * tau * (F[0] / 2.0 + prob.psi1 / tau + prob.psi0 / (tau * tau))
    if prob.nt >= 2:
        out[1] = tau * tau * (F[1] - (L @ prob.psi0) / (tau * tau))
    return out


def rhs_b(prob) -> np.ndarray:
    """b = Y f (eq. (symmetricform)), shape (n, m): time levels reversed."""
    return rhs_f(prob)[::-1].copy()


def apply_L_stencil(w: np.ndarray, d: int, N: int, tau: float, c2: float = 1.0) -> np.ndarray:
    """L w for w of shape (..., m) written as the (2d+1)-point stencil with zero
    Dirichlet values outside the grid."""
    shp = w.shape[:-1] + (N,) * d
    W = w.reshape(shp)
    h = 1.0 / (N + 1)
    lap = -2.0 * d * W
    for a in range(d):
        ax = W.ndim - 1 - a
        P = np.zeros_like(W)
        idx_dst = [slice(None)] * W.ndim
        idx_src = [slice(None)] * W.ndim
        idx_dst[ax] = slice(0, N - 1); idx_src[ax] = slice(1, N)
        P[tuple(idx_dst)] += W[tuple(idx_src)]
        idx_dst[ax] = slice(1, N); idx_src[ax] = slice(0, N - 1)
        P[tuple(idx_dst)] += W[tuple(idx_src)]
        lap = lap + P
    lap = lap / (h * h)
    return (W - 0.5 * c2 * tau * tau * lap).reshape(w.shape)


def apply_T(v: np.ndarray, d: int, N: int, tau: float, c2: float = 1.0) -> np.ndarray:
    """T v for v of shape (n, m): (T v)_i = L v_i - 2 v_{i-1} + L v_{i-2} (v_{-1} = v_{-2} = 0)."""
    Lv = apply_L_stencil(v, d, N, tau, c2)
    out = Lv.copy()
    out[1:] -= 2.0 * v[:-1]
    out[2:] += Lv[:-2]
    return out


def apply_YT(v: np.ndarray, d: int, N: int, tau: float, c2: float = 1.0) -> np.ndarray:
    """Y T v (eq. (main_system)): T v with its time levels reversed."""
    return apply_T(v, d, N, tau, c2)[::-1].copy()


def error_E(u: np.ndarray, exact_levels: np.ndarray, d: int, h: float) -> float:
    """E_{tau,h} = max_k h^{d/2} || u^(k) - u(G_h, k tau) ||_2 (Section 3)."""
    diff = u.reshape(exact_levels.shape) - exact_levels
    return float(np.max(h ** (d / 2.0) * np.linalg.norm(diff, axis=1)))


# ---------------------------------------------------------------------------
# Variable coefficient u_tt = div(a grad u) + f (Section 3, eq. (var coeff wave))
# ---------------------------------------------------------------------------

def face_coefficients(afun, d: int, N: int):
    """a sampled at the cell faces (input evaluation, from the shared input module):
    per axis ax an array with N+1 faces along ax at (f + 1/2) h, grid points elsewhere."""
    from workloads import face_coefficients as fc
    return fc(afun, d, N)


def apply_La_stencil(w: np.ndarray, faces, d: int, N: int, tau: float) -> np.ndarray:
    """L_a w = w - (tau^2/2) Delta_{a,h} w with the conservative central difference
    (Delta_{a,h} w)_i = sum_axes [a_{i+1/2}(w_{i+1} - w_i) - a_{i-1/2}(w_i - w_{i-1})] / h^2,
    a at the faces, zero Dirichlet values outside.  w has shape (..., m)."""
    h = 1.0 / (N + 1)
    shp = w.shape[:-1] + (N,) * d
    W = w.reshape(shp)
    lap = np.zeros_like(W)
    lead = W.ndim - d
    for ax in range(d):
        arr_ax = lead + (d - 1 - ax)
        pad = [(0, 0)] * W.ndim
        pad[arr_ax] = (1, 1)
        Wp = np.pad(W, pad)                                   # zeros outside
        sl = lambda a, b: tuple(slice(a, b) if k == arr_ax else slice(None) for k in range(W.ndim))
        right = Wp[sl(2, N + 2)] - W                          # w_{i+1} - w_i
        left = W - Wp[sl(0, N)]                               # w_i - w_{i-1}
        F = faces[ax]
        fsl = lambda a, b: tuple(slice(a, b) if k == (d - 1 - ax) else slice(None) for k in range(d))
        aR = F[fsl(1, N + 1)]
        aL = F[fsl(0, N)]
        lap = lap + aR * right - aL * left
    return (W - 0.5 * tau * tau * lap / (h * h)).reshape(w.shape)


def apply_YT_var(v: np.ndarray, faces, d: int, N: int, tau: float) -> np.ndarray:
    """Y T_a v with T_a the all-at-once matrix of eq. (tssystemvarwaveeq)."""
    Lv = apply_La_stencil(v, faces, d, N, tau)
    out = Lv.copy()
    out[1:] -= 2.0 * v[:-1]
    out[2:] += Lv[:-2]
    return out[::-1].copy()


def rhs_b_var(prob, faces) -> np.ndarray:
    """Y f for eq. (tssystemvarwaveeq); its second block uses L_a psi0 (the paper prints L
    there; L_a is the operator of the variable-coefficient scheme)."""
    tau = prob.tau
    F = np.array(prob.f, dtype=np.float64, copy=True)
    out = tau * tau * F
    out[0] = tau * tau * (F[0] / 2.0 + prob.psi1 / tau + prob.psi0 / (tau * tau))
    out[1] = tau * tau * F[1] - apply_La_stencil(prob.psi0, faces, prob.d, prob.N, tau)
    return out[::-1].copy()


def La_matrix(faces, d: int, N: int, tau: float) -> sp.csr_matrix:
    """L_a assembled independently of the stencil: -Delta_{a,h} = sum_axes D_ax^T diag(a_faces) D_ax / h^2
    with D_ax the (faces x points) forward-difference matrix along axis ax (Dirichlet: the
    boundary values are zero, so the first and last faces see one interior point)."""
    h = 1.0 / (N + 1)
    m = N ** d
    D1 = sp.diags([-np.ones(N), np.ones(N)], [0, -1], shape=(N + 1, N), format="csr")  # (w_i - w_{i-1}) at face i
    I = sp.identity(N, format="csr")
    A = None
    for ax in range(d):
        mats = [I] * d
        mats[d - 1 - ax] = D1
        Dk = mats[0]
        for Mx in mats[1:]:
            Dk = sp.kron(Dk, Mx, format="csr")
        term = Dk.T @ sp.diags(faces[ax].ravel()) @ Dk
        A = term if A is None else A + term
    return (sp.identity(m, format="csr") + 0.5 * tau * tau * A / (h * h)).tocsr()
