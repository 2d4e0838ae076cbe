"""P_alpha^{-1} by the paper's three-step procedure, with explicit matrices
(oracle; test infrastructure only).

Section 2.3 writes P_alpha^{-1} y = C_alpha^{-1/2} (C_alpha^{-1/2})^T y and, with
B_j = D_alpha^{-1} F^* Lambda_{alpha,j} F D_alpha and L = U Lambda U^T,
    (C_alpha^{-1/2})^T = (D^{-1} F^* (x) U)^{-T} Sigma^{-1/2} (F D (x) U^T)^{-T},
    Sigma = Lambda_{alpha,1} (x) Lambda + Lambda_{alpha,2} (x) I_m,
so (C^{-1/2})^T y is computed in three steps (Step 1: the right factor,
Step 2: the diagonal, Step 3: the left factor), and "repeating the three-step
procedure two times" gives P_alpha^{-1} y: once for (C^{-1/2})^T and once for
C^{-1/2} = (D^{-1} F^* (x) U) Sigma^{-1/2} (F D (x) U^T).

Readings of the paper adopted here (each pinned by a test):
  * F is the unitary matrix (1/sqrt(n)) [theta^{(i-1)(j-1)}], theta = exp(2 pi i/n);
    lambda_{1,k} = 1 + alpha^{2/n} theta^{2(k-1)}, lambda_{2,k} = -2 alpha^{1/n} theta^{k-1}
    (the Section 2.3 placement F^* ... F; with these eigenvalues it reproduces
    B_1, B_2 of eq. (C_decom) exactly).
  * Sigma = Lambda_{alpha,1} (x) Lambda + Lambda_{alpha,2} (x) I_m: the factor -2
    of the I-term is already inside lambda_{2,k} (as in eq. (calphaprediagform)
    and Appendix A); Step 2's extra "(-2 I_m)" is not applied a second time.
  * Sigma^{-1/2} uses the principal branch (eq. (calphasqrtdiagform)).
  * Sigma_{k,j} = Lambda_j lambda_{1,k} + lambda_{2,k} is evaluated in the algebraically
    identical form (1 - a theta^k)^2 + (Lambda_j - 1)(1 + a^2 theta^{2k}), a = alpha^{1/n},
    with 1 - a = -expm1(log(alpha)/n), 1 - cos(phi) = 2 sin^2(phi/2) and Lambda_j - 1 =
    (c^2 tau^2/2) mu_j taken directly.  The literal form loses up to ~1e-11 relative
    accuracy by cancellation when Lambda_j ~ 1 and a ~ 1 (low spatial modes, large n);
    the rewritten form is pinned against the literal formula in 50-digit arithmetic.
  * U = S (x) ... (x) S with S the orthonormal DST-I matrix (Section 2.3: on a
    uniform grid U is the multi-dimensional discrete sine transform).
No FFT is used: every transform is an explicit matrix product.
"""
from __future__ import annotations

import numpy as np


def dst_matrix(N: int) -> np.ndarray:
    """Orthonormal DST-I matrix S_{jk} = sqrt(2/(N+1)) sin(pi j k/(N+1)), j,k = 1..N
    (symmetric and its own inverse)."""
    j = np.arange(1, N + 1, dtype=np.float64)
    return np.sqrt(2.0 / (N + 1)) * np.sin(np.pi * np.outer(j, j) / (N + 1))


def laplacian_eigenvalues_1d(N: int) -> np.ndarray:
    """Eigenvalues of -Delta_h in 1D for the eigenvectors S[:, k-1]:
    mu_k = (4/h^2) sin^2(k pi h / 2), k = 1..N."""
    h = 1.0 / (N + 1)
    k = np.arange(1, N + 1, dtype=np.float64)
    return 4.0 / (h * h) * np.sin(k * np.pi * h / 2.0) ** 2


def L_eigenvalues_minus_one(d: int, N: int, tau: float, c2: float = 1.0) -> np.ndarray:
    """Lambda - 1 = (c^2 tau^2/2) * (eigenvalues of -Delta_h), lexicographic order of
    the columns of U = S (x) ... (x) S, shape (m,)."""
    mu = laplacian_eigenvalues_1d(N)
    tot = np.zeros((N,) * d)
    for a in range(d):
        shp = [1] * d
        shp[d - 1 - a] = N
        tot = tot + mu.reshape(shp)
    return (0.5 * c2 * tau * tau * tot).ravel()


def L_eigenvalues(d: int, N: int, tau: float, c2: float = 1.0) -> np.ndarray:
    """Lambda: eigenvalues of L = I - (c^2 tau^2/2) Delta_h in the lexicographic
    order of the columns of U = S (x) ... (x) S, shape (m,)."""
    return 1.0 + L_eigenvalues_minus_one(d, N, tau, c2)


def theta_pow(e, n: int) -> np.ndarray:
    """theta_n^e = exp(2 pi i e / n) for integer arrays e: the exponent is reduced
    mod n exactly and the angle functions are evaluated in extended precision
    (numpy longdouble), then rounded to complex128."""
    e = np.mod(np.asarray(e, dtype=np.int64), n)
    ld = np.longdouble
    ang = ld(2) * ld(np.pi) * e.astype(ld) / ld(n)
    # long-double pi: refine numpy's double pi by one correction term
    ang = ang + ld(2) * (ld("3.14159265358979323846264338327950288") - ld(np.pi)) * e.astype(ld) / ld(n)
    return (np.cos(ang).astype(np.float64) + 1j * np.sin(ang).astype(np.float64))


def fourier_matrix(n: int) -> np.ndarray:
    """Unitary F = (1/sqrt(n)) [theta_n^{(i-1)(j-1)}], theta_n = exp(2 pi i / n)."""
    i = np.arange(n)
    return theta_pow(np.outer(i, i), n) / np.sqrt(n)


def D_alpha_diag(n: int, alpha: float) -> np.ndarray:
    """Diagonal of D_alpha = diag(alpha^{(i-1)/n}), i = 1..n."""
    return alpha ** (np.arange(n, dtype=np.float64) / n)


def Lambda_alpha(n: int, alpha: float):
    """lambda_{1,k} = 1 + alpha^{2/n} theta^{2(k-1)}, lambda_{2,k} = -2 alpha^{1/n} theta^{k-1}."""
    k = np.arange(n)
    theta_k = theta_pow(k, n)
    lam1 = 1.0 + alpha ** (2.0 / n) * theta_pow(2 * k, n)
    lam2 = -2.0 * alpha ** (1.0 / n) * theta_k
    return lam1, lam2


def Sigma_literal(n: int, alpha: float, Lam: np.ndarray) -> np.ndarray:
    """Diagonal of Lambda_{alpha,1} (x) Lambda + Lambda_{alpha,2} (x) I_m as an (n, m)
    array, written exactly as the product and sum of the definitions."""
    lam1, lam2 = Lambda_alpha(n, alpha)
    return lam1[:, None] * Lam[None, :] + lam2[:, None]


def Sigma(n: int, alpha: float, Lam_minus_one: np.ndarray) -> np.ndarray:
    """The same diagonal evaluated without cancellation:
    Sigma_{k,j} = (1 - a theta^k)^2 + (Lambda_j - 1)(1 + a^2 theta^{2k}), a = alpha^{1/n}
    (expand the square: 1 - 2 a theta + a^2 theta^2 + (Lambda - 1)(1 + a^2 theta^2)
    = Lambda (1 + a^2 theta^2) - 2 a theta)."""
    la = np.log(alpha) / n
    one_minus_a = -np.expm1(la)
    a = np.exp(la)
    k = np.arange(n)
    th = theta_pow(k, n)                              # theta^k
    s_half = theta_pow(k, 2 * n).imag                 # sin(phi/2), phi = 2 pi k/n
    wr = one_minus_a + 2.0 * a * s_half * s_half      # Re(1 - a theta^k) = (1-a) + a (1 - cos phi)
    wi = -a * th.imag                                 # Im(1 - a theta^k)
    w2 = (wr - wi) * (wr + wi) + 2j * wr * wi         # (1 - a theta^k)^2
    qr = one_minus_a * (1.0 + a) + 2.0 * a * a * th.real ** 2   # 1 + a^2 cos(2 phi)
    q = qr + 1j * a * a * theta_pow(2 * k, n).imag    # 1 + a^2 theta^{2k}
    return w2[:, None] + Lam_minus_one[None, :] * q[:, None]


def apply_space(X: np.ndarray, S: np.ndarray, d: int, N: int) -> np.ndarray:
    """(I_n (x) U) X with U = S (x) ... (x) S applied to every time level of X (n, m)."""
    n = X.shape[0]
    Y = X.reshape((n,) + (N,) * d)
    for a in range(d):
        ax = d - a  # array axis of spatial direction a (x is last)
        Y = np.moveaxis(np.tensordot(Y, S, axes=([ax], [1])), -1, ax)
    return Y.reshape(X.shape)


class ABACPreconditioner:
    """Applies P_alpha^{-1} = C_alpha^{-1/2} (C_alpha^{-1/2})^T by Section 2.3's
    three steps, done twice, with explicit F, D_alpha and DST matrices."""

    def __init__(self, d: int, N: int, n: int, tau: float, alpha: float, c2: float = 1.0):
        self.d, self.N, self.n, self.alpha = d, N, n, alpha
        self.S = dst_matrix(N)                      # U = S (x) .. (x) S, U = U^T = U^{-1}
        self.Lam_m1 = L_eigenvalues_minus_one(d, N, tau, c2)
        self.Lam = 1.0 + self.Lam_m1
        F = fourier_matrix(n)
        dg = D_alpha_diag(n, alpha)
        FD = F * dg[None, :]                        # F D_alpha
        DinvFs = (1.0 / dg)[:, None] * F.conj().T   # D_alpha^{-1} F^*  (F is unitary)
        # (F D)^{-1} = D^{-1} F^* and (D^{-1} F^*)^{-1} = F D, since F F^* = I
        self.time_step1_T = DinvFs.T                # time part of (F D (x) U^T)^{-T}
        self.time_step3_T = FD.T                    # time part of (D^{-1} F^* (x) U)^{-T}
        self.time_right = FD                        # right factor of C^{-1/2}
        self.time_left = DinvFs                     # left factor of C^{-1/2}
        Sig = Sigma(n, alpha, self.Lam_m1)
        self.Sigma = Sig
        self.g = 1.0 / np.sqrt(Sig)                 # principal branch: Sigma^{-1/2}

    def _kron_apply(self, At: np.ndarray, X: np.ndarray) -> np.ndarray:
        """(At (x) U) X for X of shape (n, m): time factor At, space factor U (= U^T)."""
        Xs = apply_space(X.real, self.S, self.d, self.N)
        if np.iscomplexobj(X):
            Xs = Xs + 1j * apply_space(X.imag, self.S, self.d, self.N)
        return At @ Xs

    def apply_Cinvsqrt_T(self, y: np.ndarray) -> np.ndarray:
        """(C_alpha^{-1/2})^T y: Step 1, Step 2, Step 3 of Section 2.3."""
        yt = self._kron_apply(self.time_step1_T, y)      # Step 1
        zt = self.g * yt                                  # Step 2 (transpose of a diagonal)
        return self._kron_apply(self.time_step3_T, zt)   # Step 3

    def apply_Cinvsqrt(self, y: np.ndarray) -> np.ndarray:
        """C_alpha^{-1/2} y = (D^{-1} F^* (x) U) Sigma^{-1/2} (F D (x) U^T) y."""
        yt = self._kron_apply(self.time_right, y)
        zt = self.g * yt
        return self._kron_apply(self.time_left, zt)

    def apply(self, y: np.ndarray, return_imag: bool = False):
        """P_alpha^{-1} y for y of shape (n, m); the imaginary residue (zero in exact
        arithmetic, Lemma real_C_alpha) is discarded, or returned on request."""
        z = self.apply_Cinvsqrt(self.apply_Cinvsqrt_T(y.astype(np.complex128)))
        if return_imag:
            return z.real.copy(), z.imag.copy()
        return z.real.copy()

    def apply_C(self, v: np.ndarray) -> np.ndarray:
        """C_alpha v via its diagonalisation (used for invariant checks)."""
        yt = self._kron_apply(self.time_right, v.astype(np.complex128))
        return self._kron_apply(self.time_left, self.Sigma * yt).real.copy()


def apply_C_alpha_direct(v: np.ndarray, d: int, N: int, tau: float, alpha: float,
                         c2: float = 1.0) -> np.ndarray:
    """C_alpha v straight from def. (matrix_C_alpha): T v plus the wrap-around
    blocks (block row 1: alpha L v_{n-1} - 2 alpha v_n; block row 2: alpha L v_n)."""
    from .system import apply_T, apply_L_stencil
    out = apply_T(v, d, N, tau, c2)
    n = v.shape[0]
    Lv_last = apply_L_stencil(v[n - 1], d, N, tau, c2)
    Lv_prev = apply_L_stencil(v[n - 2], d, N, tau, c2)
    out[0] += alpha * Lv_prev - 2.0 * alpha * v[n - 1]
    out[1] += alpha * Lv_last
    return out


def time_part_modes(d: int, N: int, n: int, tau: float, alpha: float, Yh: np.ndarray, modes,
                    c2: float = 1.0) -> np.ndarray:
    """(I_n (x) U) P_alpha^{-1} (I_n (x) U) restricted to chosen spatial modes.

    Yh (n, len(modes)) holds the DST-basis time series of the modes listed in `modes`
    (column indices of U).  Writing P_alpha^{-1} = C^{-1/2} (C^{-1/2})^T with the
    factors of Section 2.3 and using U U = I between them, the DST-basis map acts on
    the time series of mode j alone:
        z_j = (D^{-1} F^*) G_j (F D)(F D)^T G_j (D^{-1} F^*)^T y_j,
    G_j = diag_k Sigma_{k,j}^{-1/2} (the time factors of Steps 1-3, twice).  Only the
    Sigma columns of the chosen modes are formed, so any grid size can be sampled."""
    Lam_m1 = L_eigenvalues_minus_one(d, N, tau, c2)[np.asarray(modes)]
    g = 1.0 / np.sqrt(Sigma(n, alpha, Lam_m1))       # (n, len(modes)), principal branch
    F = fourier_matrix(n)
    dg = D_alpha_diag(n, alpha)
    FD = F * dg[None, :]
    DinvFs = (1.0 / dg)[:, None] * F.conj().T
    a = g * (DinvFs.T @ Yh.astype(np.complex128))   # (C^{-1/2})^T: Steps 1 and 2
    c = g * (FD @ (FD.T @ a))                        # its Step 3, then C^{-1/2}'s right factor and diagonal
    return (DinvFs @ c).real.copy()                  # C^{-1/2}'s left factor
