"""Pins for the CPU oracle against what the paper and the mathematics fix
(closed forms, invariants, printed values, library special cases, brute force).
No GPU needed."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import workloads as W
from oracle import dense as D
from oracle import fast as F
from oracle import minres as M
from oracle import stepping as ST
from oracle import system as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,alpha", [(4, 0.3), (8, 1e-2), (16, 1e-6), (7, 0.5)])
def test_B_alpha_diagonalisation(n, alpha):
    """B_j = D^{-1} F^* Lambda_j F D (Section 2.3) reproduces B_1, B_2 of eq. (C_decom)
    written entry by entry; the other placement (F ... F^*) with the same
    eigenvalues does not (so the test distinguishes the two readings)."""
    B1, B2 = S.B_alpha(n, alpha)
    Fm = F.fourier_matrix(n)
    dg = F.D_alpha_diag(n, alpha)
    l1, l2 = F.Lambda_alpha(n, alpha)
    rec1 = (np.diag(1 / dg) @ Fm.conj().T @ np.diag(l1) @ Fm @ np.diag(dg))
    rec2 = (np.diag(1 / dg) @ Fm.conj().T @ np.diag(l2) @ Fm @ np.diag(dg))
    tol = max(1e-12, 1e-14 / alpha)   # D_alpha^{-1} amplifies round-off by ~1/alpha
    assert np.abs(rec1 - B1).max() < tol
    assert np.abs(rec2 - (-2.0) * B2).max() < tol
    other = np.diag(1 / dg) @ Fm @ np.diag(l2) @ Fm.conj().T @ np.diag(dg)
    assert np.abs(other - (-2.0) * B2).max() > 1e-3


def test_fourier_unitary_and_D():
    n = 12
    Fm = F.fourier_matrix(n)
    assert np.abs(Fm @ Fm.conj().T - np.eye(n)).max() < 1e-13
    assert np.abs(Fm - Fm.T).max() < 1e-15
    dg = F.D_alpha_diag(n, 1e-3)
    assert dg[0] == 1.0 and abs(dg[-1] - 1e-3 ** ((n - 1) / n)) < 1e-15


@pytest.mark.parametrize("d,N,n", [(1, 5, 6), (2, 3, 4), (1, 4, 3), (2, 3, 2)])
def test_C_alpha_definition_equals_split(d, N, n):
    """def. (matrix_C_alpha) written block by block == B_1 (x) L + B_2 (x) (-2I) (eq. C_decom)."""
    L = S.L_matrix(d, N, 1.0 / n)
    for alpha in (0.0, 0.25, 1.0):
        A = S.C_alpha_matrix(L, n, alpha).toarray()
        B = S.C_alpha_from_split(L, n, alpha).toarray()
        assert np.abs(A - B).max() < 1e-14
    # alpha = 0 gives T itself (Appendix A)
    assert np.abs(S.C_alpha_matrix(L, n, 0.0).toarray() - S.T_matrix(L, n).toarray()).max() == 0.0


@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_laplacian_1d_closed_form(N):
    """Eigenvalues of the 3-point Dirichlet Laplacian: -(4/h^2) sin^2(k pi h/2)."""
    ev = np.sort(np.linalg.eigvalsh(S.laplacian_1d(N).toarray()))
    cf = np.sort(-F.laplacian_eigenvalues_1d(N))
    assert np.allclose(ev, cf, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("d,N", [(1, 7), (2, 5), (3, 3), (2, 4)])
def test_dst_diagonalises_L(d, N):
    """S is symmetric orthonormal and U^T L U = diag(Lambda) with U = S (x)..(x) S
    in lexicographic order (Section 2.3, U = multi-dimensional DST)."""
    Sm = F.dst_matrix(N)
    assert np.abs(Sm @ Sm - np.eye(N)).max() < 1e-13
    assert np.abs(Sm - Sm.T).max() == 0.0
    tau = 0.37
    L = S.L_matrix(d, N, tau, c2=1.7).toarray()
    U = Sm
    for _ in range(d - 1):
        U = np.kron(U, Sm)
    Lam = F.L_eigenvalues(d, N, tau, c2=1.7)
    assert np.abs(U.T @ L @ U - np.diag(Lam)).max() < 1e-11 * np.abs(Lam).max()
    assert Lam.min() > 1.0  # sigma(L) in (1, inf)


@pytest.mark.parametrize("d,N,n,alpha", [(1, 5, 8, 1e-2), (2, 3, 4, 0.3), (1, 3, 6, 0.9)])
def test_Sigma_is_spectrum_of_C_alpha(d, N, n, alpha):
    """The diagonal Sigma = Lambda_1 (x) Lambda + Lambda_2 (x) I equals the spectrum of the
    dense C_alpha (eq. calphaprediagform; Appendix A); and every eigenvalue lies off
    (-inf, 0] (Lemma calphanonsinglm)."""
    tau = 1.0 / n
    L = S.L_matrix(d, N, tau)
    C = S.C_alpha_matrix(L, n, alpha).toarray()
    ev = np.linalg.eigvals(C)
    Sig = F.Sigma(n, alpha, F.L_eigenvalues_minus_one(d, N, tau)).ravel()
    # match as multisets
    used = np.zeros(len(ev), bool)
    for s in Sig:
        dist = np.abs(ev - s) + used * 1e300
        k = np.argmin(dist)
        assert dist[k] < 1e-9 * max(1.0, abs(s))
        used[k] = True
    assert not np.any((np.abs(Sig.imag) < 1e-14) & (Sig.real <= 0))


@pytest.mark.parametrize("n,alpha,tau,N", [(1024, 0.1, 1 / 1024, 63), (256, 1e-6, 1 / 256, 255),
                                            (64, 1e-3, 1 / 64, 63), (512, 1e-2, 1 / 512, 511),
                                            (128, 1.0, 1 / 128, 127)])
def test_sigma_cancellation_free_form(n, alpha, tau, N):
    """Sigma = (1 - a theta)^2 + (Lambda - 1)(1 + a^2 theta^2) equals the literal
    Lambda lambda_1 + lambda_2 evaluated in 50-digit arithmetic (mpmath) to 1e-14
    relative (plus a few ulps of the terms' size, which matters only at alpha = 1),
    at sample points including the lowest modes where the literal FP64 formula cancels."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    lm1 = F.L_eigenvalues_minus_one(1, N, tau)
    Sig = F.Sigma(n, alpha, lm1)
    h = mp.mpf(1) / (N + 1)
    worst = 0.0
    for k in [0, 1, 2, n // 4, n // 2 - 1, n // 2, n - 1]:
        for j in [0, 1, N // 2, N - 1]:
            mu = 4 / h ** 2 * mp.sin((j + 1) * mp.pi * h / 2) ** 2
            lam = 1 + mp.mpf(tau) ** 2 / 2 * mu
            a = mp.power(mp.mpf(alpha), mp.mpf(1) / n)
            th = mp.exp(2j * mp.pi * k / n)
            exact = lam * (1 + a * a * th * th) - 2 * a * th
            # size of the two terms of the rewritten form: at alpha = 1 they can cancel
            # for real (the ABC near-singularity), so allow a few ulps of that size
            scale = abs((1 - a * th) ** 2) + abs((lam - 1) * (1 + a * a * th * th))
            err = float(abs(Sig[k, j] - complex(exact)))
            worst = max(worst, err / float(1e-14 * abs(exact) + 4e-16 * scale))
    assert worst <= 1.0, worst


def test_appendix_A_eigenvalue_form():
    """Appendix A's real/imaginary split of mu = lambda lambda_1k + lambda_2k."""
    n, alpha, lam = 16, 1e-3, 3.7
    l1, l2 = F.Lambda_alpha(n, alpha)
    mu = lam * l1 + l2
    a = alpha ** (1.0 / n)
    w = 2 * np.pi * np.arange(n) / n
    re = lam * (1 - a * a) + 2 * a * np.cos(w) * (lam * a * np.cos(w) - 1)
    im = 2 * a * np.sin(w) * (lam * a * np.cos(w) - 1)
    assert np.allclose(mu.real, re, atol=1e-13) and np.allclose(mu.imag, im, atol=1e-13)


@pytest.mark.parametrize("d,N,n", [(1, 5, 8), (2, 3, 4), (3, 2, 4)])
def test_stencil_operators_against_sparse(d, N, n):
    """Y T v by stencil == sparse Y T (eq. main_system); Y T is symmetric; Y^2 = I;
    C_alpha applied from its definition and through its diagonalisation agree."""
    tau = 1.0 / n
    L = S.L_matrix(d, N, tau, c2=2.0)
    T = S.T_matrix(L, n)
    Y = S.Y_matrix(n, N ** d)
    YT = (Y @ T).toarray()
    assert np.abs(YT - YT.T).max() == 0.0
    assert np.abs((Y @ Y).toarray() - np.eye(n * N ** d)).max() == 0.0
    v = _rng(3).standard_normal((n, N ** d))
    assert np.abs(S.apply_YT(v, d, N, tau, 2.0).ravel() - YT @ v.ravel()).max() < 1e-12
    alpha = 0.2
    C = S.C_alpha_matrix(S.L_matrix(d, N, tau, 1.0), n, alpha).toarray()
    assert np.abs(F.apply_C_alpha_direct(v, d, N, tau, alpha).ravel() - C @ v.ravel()).max() < 1e-12
    pc = F.ABACPreconditioner(d, N, n, tau, alpha)
    assert np.abs(pc.apply_C(v).ravel() - C @ v.ravel()).max() < 1e-12


# --------------------------------------------------------------------------
# square roots, P_alpha, the fast three-step inverse
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d,N,n,alpha", [(1, 5, 8, 1e-1), (1, 7, 16, 1e-3), (2, 3, 8, 1e-2)])
def test_sqrt_C_alpha_properties(d, N, n, alpha):
    """Schur and eigendecomposition square roots agree, square to C_alpha, are real
    and Y C^{1/2} is symmetric (Lemma real_C_alpha); P_alpha is SPD (def. matrix_P)."""
    tau = 1.0 / n
    C = S.C_alpha_matrix(S.L_matrix(d, N, tau), n, alpha).toarray()
    R1 = D.sqrtm_schur(C)
    R2 = D.sqrtm_eig(C)
    sc = np.abs(R1).max()
    assert np.abs(R1 - R2).max() < 1e-9 * sc
    assert np.abs(R2.imag).max() < 1e-9 * sc
    assert np.abs(R1 @ R1 - C).max() < 1e-10 * np.abs(C).max()
    Y = S.Y_matrix(n, N ** d).toarray()
    YR = Y @ R1.real
    assert np.abs(YR - YR.T).max() < 1e-10 * sc
    P = D.P_alpha_dense(C).real
    assert np.abs(P - P.T).max() < 1e-10 * np.abs(P).max()
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0.0


@pytest.mark.parametrize("d,N,n", [(1, 7, 16), (2, 3, 8), (2, 7, 8), (1, 15, 32)])
@pytest.mark.parametrize("alpha,tol", [(1e-1, 1e-12), (1e-2, 1e-12), (1e-3, 1e-12), (1e-6, 1e-9)])
def test_fast_prec_equals_dense_cholesky(d, N, n, alpha, tol):
    """Section 2.3's three-step procedure (done twice) == Cholesky solve with the dense
    P_alpha = (sqrtm C_alpha)^T sqrtm C_alpha."""
    tau = 1.0 / n
    C = S.C_alpha_matrix(S.L_matrix(d, N, tau), n, alpha).toarray()
    P = D.P_alpha_dense(C).real
    pc = F.ABACPreconditioner(d, N, n, tau, alpha)
    v = _rng(5).standard_normal((n, N ** d))
    z1, zi = pc.apply(v, return_imag=True)
    z2 = D.prec_solve_dense(P, v.ravel())
    assert np.abs(z1.ravel() - z2).max() / np.abs(z2).max() < tol
    assert np.abs(zi).max() < 1e3 * tol * np.abs(z1).max()   # Lemma real_C_alpha


@pytest.mark.parametrize("d,N,n,alpha", [(1, 63, 64, 1e-2), (2, 15, 32, 1e-3), (3, 7, 16, 1e-1),
                                         (2, 31, 16, 1e-6)])
def test_Q_alpha_involution_and_symmetry(d, N, n, alpha):
    """(P^{-1} Y C_alpha)^2 = I (Lemma qalphaorthoglm: Q_alpha orthogonal and symmetric)
    and <P^{-1} x, y> = <x, P^{-1} y>, matrix-free at moderate sizes."""
    tau = 1.0 / n
    pc = F.ABACPreconditioner(d, N, n, tau, alpha)
    v = _rng(7).standard_normal((n, N ** d))
    def Q(x):
        return pc.apply(F.apply_C_alpha_direct(x, d, N, tau, alpha)[::-1].copy())
    w = Q(Q(v))
    tol = max(1e-12, 1e-13 / alpha)   # round-off grows like eps / alpha (D_alpha^{-1})
    assert np.abs(w - v).max() / np.abs(v).max() < tol
    x, y = _rng(8).standard_normal((2, n, N ** d))
    a, b = np.vdot(pc.apply(x), y), np.vdot(x, pc.apply(y))
    assert abs(a - b) / abs(a) < tol
    assert np.vdot(pc.apply(x), x) > 0


def test_alpha_one_is_abc_preconditioner():
    """alpha = 1: P_1 = (C_1^{1/2})^T C_1^{1/2} = |C_1| (Remark p1badpermformremark),
    and the fast procedure gives |C_1|^{-1}."""
    d, N, n = 1, 4, 6
    tau = 1.0 / n
    C = S.C_alpha_matrix(S.L_matrix(d, N, tau), n, 1.0).toarray()
    Sig = F.Sigma(n, 1.0, F.L_eigenvalues_minus_one(d, N, tau))
    assert np.abs(Sig).min() > 1e-3 and not np.any((np.abs(Sig.imag) < 1e-12) & (Sig.real <= 0))
    P1 = D.P_alpha_dense(C).real
    A = D.abs_sym(C)
    assert np.abs(P1 - A).max() < 1e-10 * np.abs(A).max()
    pc = F.ABACPreconditioner(d, N, n, tau, 1.0)
    v = _rng(9).standard_normal((n, N))
    assert np.abs(pc.apply(v).ravel() - np.linalg.solve(A, v.ravel())).max() < 1e-10


def test_R_alpha_norm_and_spectrum_enclosure():
    """||R_alpha||_2 = alpha (sqrt(||L||^2 + 1) + 1) (proof of Lemma precedmatspectrmlm) and
    sigma(P^{-1} Y T) within +-1 +- ||C^{-1/2}||^2 ||R_alpha|| (inequality ralphaesti1 +
    Lemma eigenperturblm)."""
    d, N, n = 1, 7, 16
    tau = 1.0 / n
    Ls = S.L_matrix(d, N, tau)
    T = S.T_matrix(Ls, n).toarray()
    Y = S.Y_matrix(n, N).toarray()
    nL = np.linalg.norm(Ls.toarray(), 2)
    for alpha in (0.5, 0.1, 1e-2, 1e-3):
        C = S.C_alpha_matrix(Ls, n, alpha).toarray()
        R = C - T
        assert abs(np.linalg.norm(R, 2) - alpha * (np.sqrt(nL ** 2 + 1) + 1)) < 1e-10 * np.linalg.norm(R, 2)
        Ci = np.linalg.inv(D.sqrtm_schur(C).real)
        bound = np.linalg.norm(Ci, 2) ** 2 * np.linalg.norm(R, 2)
        P = D.P_alpha_dense(C).real
        ev = np.linalg.eigvals(np.linalg.solve(P, Y @ T))
        assert np.abs(ev.imag).max() < 1e-8
        assert np.max(np.abs(np.abs(ev.real) - 1.0)) <= bound * (1 + 1e-8)


def test_ideal_preconditioner_two_eigenvalues_and_two_steps():
    """Proposition ideal_P: ((T^{1/2})^T T^{1/2})^{-1} Y T has only the eigenvalues +-1, so
    MINRES converges in two iterations."""
    d, N, n = 1, 5, 8
    tau = 1.0 / n
    T = S.T_matrix(S.L_matrix(d, N, tau), n).toarray()
    Y = S.Y_matrix(n, N).toarray()
    Pid = D.ideal_preconditioner(T)
    ev = np.linalg.eigvals(np.linalg.solve(Pid, Y @ T))
    assert np.max(np.abs(np.abs(ev) - 1.0)) < 1e-9
    b = _rng(10).standard_normal(n * N)
    x, info = M.minres(lambda v: Y @ T @ v, lambda v: np.linalg.solve(Pid, v), b, rtol=1e-10)
    assert info["iters"] <= 2


# --------------------------------------------------------------------------
# MINRES
# --------------------------------------------------------------------------

def test_minres_iterates_minimise_over_krylov_space():
    """Brute force: the k-th iterate minimises ||b - A x||_{P^{-1}} over
    x in K_k(P^{-1} A, P^{-1} b)."""
    d, N, n, alpha = 1, 3, 8, 0.3
    tau = 1.0 / n
    T = S.T_matrix(S.L_matrix(d, N, tau), n).toarray()
    Y = S.Y_matrix(n, N).toarray()
    A = Y @ T
    P = D.P_alpha_dense(S.C_alpha_matrix(S.L_matrix(d, N, tau), n, alpha).toarray()).real
    Pi = np.linalg.inv(P)
    Pih = sla.sqrtm(Pi).real
    b = _rng(11).standard_normal(n * N)
    for k in range(1, 6):
        x, info = M.minres(lambda v: A @ v, lambda v: Pi @ v, b, rtol=0.0, maxit=k)
        assert info["iters"] == k
        K = [Pi @ b]
        for _ in range(k - 1):
            K.append(Pi @ A @ K[-1])
        Kq, _ = np.linalg.qr(np.array(K).T)
        c, *_ = np.linalg.lstsq(Pih @ A @ Kq, Pih @ b, rcond=None)
        xb = Kq @ c
        assert np.linalg.norm(x - xb) < 1e-9 * np.linalg.norm(xb)
        # and the recurrence estimate is the P^{-1}-norm of the true residual
        r = b - A @ x
        assert abs(np.sqrt(r @ Pi @ r) / np.sqrt(b @ Pi @ b) - info["relres_est"]) < 1e-9


def test_minres_matches_scipy():
    """Library special case: scipy.sparse.linalg.minres with the same preconditioner."""
    d, N, n, alpha = 2, 7, 16, 1e-3
    tau = 1.0 / n
    pc = F.ABACPreconditioner(d, N, n, tau, alpha)
    b = _rng(12).standard_normal((n, N * N))
    A = lambda v: S.apply_YT(v.reshape(n, -1), d, N, tau).ravel()
    Aop = spla.LinearOperator((b.size, b.size), matvec=A)
    Mop = spla.LinearOperator((b.size, b.size), matvec=lambda v: pc.apply(v.reshape(n, -1)).ravel())
    xs, _ = spla.minres(Aop, b.ravel(), M=Mop, rtol=1e-13, maxiter=200)
    x, info = M.minres(lambda v: S.apply_YT(v, d, N, tau), pc.apply, b, rtol=1e-12)
    assert np.linalg.norm(x.ravel() - xs) < 1e-9 * np.linalg.norm(xs)


def test_minres_residual_bound_lemma():
    """Lemma minrescvglm: ||r_k||_2 <= 2 ((sqrt(a1 a4) - sqrt(a2 a3))/(sqrt(a1 a4) + sqrt(a2 a3)))^{floor(k/2)} ||r_0||_2
    with r_k = P^{-1}(y - A x_k) and the spectrum of P^{-1}A inside [-a1,-a2] u [a3,a4]."""
    d, N, n, alpha = 1, 7, 16, 0.2
    tau = 1.0 / n
    T = S.T_matrix(S.L_matrix(d, N, tau), n).toarray()
    A = S.Y_matrix(n, N).toarray() @ T
    P = D.P_alpha_dense(S.C_alpha_matrix(S.L_matrix(d, N, tau), n, alpha).toarray()).real
    ev = np.linalg.eigvals(np.linalg.solve(P, A)).real
    neg, pos = -ev[ev < 0], ev[ev > 0]
    a1, a2, a3, a4 = neg.max(), neg.min(), pos.min(), pos.max()
    ln = max(a1 - a2, a4 - a3)
    a2, a3 = a1 - ln, a4 - ln       # equal-length enclosing intervals
    assert a2 > 0 and a3 > 0
    rho = (np.sqrt(a1 * a4) - np.sqrt(a2 * a3)) / (np.sqrt(a1 * a4) + np.sqrt(a2 * a3))
    b = _rng(13).standard_normal(n * N)
    r0 = np.linalg.norm(np.linalg.solve(P, b))
    for k in range(1, 12):
        x, _ = M.minres(lambda v: A @ v, lambda v: np.linalg.solve(P, v), b, rtol=0.0, maxit=k)
        rk = np.linalg.norm(np.linalg.solve(P, b - A @ x))
        assert rk <= 2 * rho ** (k // 2) * r0 * (1 + 1e-9) + 1e-13


# --------------------------------------------------------------------------
# the scheme: sequential stepping, Table 2, convergence order, flat iterations
# --------------------------------------------------------------------------

def test_all_at_once_equals_sequential_stepping():
    """The all-at-once solution (dense solve of T u = f) == sequential stepping; and the
    oracle MINRES solution agrees to 1e-12."""
    p = W.config_2d(N=7, nt=16, seed=21)
    from oracle.system import L_matrix, T_matrix, rhs_f, rhs_b
    f = rhs_f(p)
    T = T_matrix(L_matrix(2, 7, p.tau), 16).toarray()
    u_dense = np.linalg.solve(T, f.ravel()).reshape(f.shape)
    u_seq = ST.sequential_solve(p)
    assert np.abs(u_dense - u_seq).max() < 1e-12 * np.abs(u_dense).max()
    pc = F.ABACPreconditioner(2, 7, 16, p.tau, 1e-6)
    x, info = M.minres(lambda v: S.apply_YT(v, 2, 7, p.tau), pc.apply, rhs_b(p), rtol=1e-14, maxit=50)
    assert np.abs(x - u_seq).max() < 1e-12 * np.abs(u_seq).max()


def _table(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _table("table2_example1.txt"), ids=lambda r: f"tau2^-{int(r[0])}_h2^-{int(r[1])}")
def test_table2_exact_discrete_errors(row):
    """Table 2, MINRES-P_1 column (~ exact discrete solution): E_{tau,h} of the scheme's
    exact solution (sequential stepping) within 1% for all 16 (tau, h); the DoF column
    n (1/h - 1)^2 checks too."""
    lt, lh, dof, e_pa, e_p1, e_i = row
    nt, N = 2 ** int(lt), 2 ** int(lh) - 1
    assert nt * N * N == int(dof)
    p = W.example1(N, nt)
    u = ST.sequential_solve(p)
    E = S.error_E(u, p.exact_levels(), 2, p.h)
    assert abs(E - e_p1) <= 0.01 * e_p1


@pytest.mark.parametrize("row", [r for r in _table("table2_example1.txt") if r[1] <= 5 or (r[0] <= 5 and r[1] <= 6)],
                         ids=lambda r: f"tau2^-{int(r[0])}_h2^-{int(r[1])}")
def test_table1_table2_minres_P_alpha(row):
    """Tables 1 and 2, MINRES-P_alpha columns: alpha = 1e-6, zero initial guess, relative
    residual tolerance 1e-6 -> 2 iterations and the printed E_{tau,h} (within 1%)."""
    lt, lh, dof, e_pa, e_p1, e_i = row
    nt, N = 2 ** int(lt), 2 ** int(lh) - 1
    p = W.example1(N, nt, alpha=1e-6)
    pc = F.ABACPreconditioner(2, N, nt, p.tau, 1e-6)
    x, info = M.minres(lambda v: S.apply_YT(v, 2, N, p.tau), pc.apply, S.rhs_b(p), rtol=1e-6)
    assert info["iters"] == 2
    E = S.error_E(x, p.exact_levels(), 2, p.h)
    assert abs(E - e_pa) <= 0.01 * e_pa


def test_second_order_convergence_manufactured():
    """Noise-free 1D twin of the 1D config: E = O(tau^2 + h^2), ratio ~4 per halving."""
    errs = []
    for N, nt in [(15, 16), (31, 32), (63, 64), (127, 128)]:
        p = W.config_1d(N=N, nt=nt, noise=0.0)
        u = ST.sequential_solve(p)
        errs.append(S.error_E(u, p.exact_levels(), 1, p.h))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios


def test_iteration_counts_flat_in_size():
    """Theorem maincvgthm: iteration counts independent of tau and h (alpha = 1e-6,
    true relative residual 1e-8)."""
    its = []
    for N, nt in [(15, 16), (31, 32), (63, 64), (127, 128), (255, 256)]:
        p = W.config_1d(N=N, nt=nt)
        pc = F.ABACPreconditioner(1, N, nt, p.tau, 1e-6)
        _, info = M.minres(lambda v: S.apply_YT(v, 1, N, p.tau), pc.apply, S.rhs_b(p), rtol=1e-8)
        its.append(info["iters"])
    for N, nt in [(7, 8), (15, 16), (31, 32)]:
        p = W.config_2d(N=N, nt=nt)
        pc = F.ABACPreconditioner(2, N, nt, p.tau, 1e-6)
        _, info = M.minres(lambda v: S.apply_YT(v, 2, N, p.tau), pc.apply, S.rhs_b(p), rtol=1e-8)
        its.append(info["iters"])
    assert max(its) - min(its) <= 2 and max(its) <= 8, its


def test_error_metric_closed_form():
    """E_{tau,h} of a constant offset c on every level = h^{d/2} c sqrt(m)."""
    N, d, n = 9, 2, 4
    ex = np.zeros((n, N * N))
    u = ex + 0.5
    h = 1.0 / (N + 1)
    assert abs(S.error_E(u, ex, d, h) - h * 0.5 * N) < 1e-15


@pytest.mark.parametrize("d,N,n,alpha,c2", [(1, 15, 16, 1e-2, 1.0), (2, 7, 8, 1e-3, 1.7), (3, 3, 8, 0.3, 0.5)])
def test_time_part_modes_equals_full_preconditioner(d, N, n, alpha, c2):
    """The sampled DST-basis time map equals (I (x) U) P^{-1} (I (x) U) computed with the
    full three-step procedure (explicit DSTs), on every mode and on a subset."""
    tau = 1.0 / n
    m = N ** d
    rng = np.random.default_rng(5)
    Yh = rng.standard_normal((n, m))
    pc = F.ABACPreconditioner(d, N, n, tau, alpha, c2=c2)
    S = F.dst_matrix(N)
    full = F.apply_space(pc.apply(F.apply_space(Yh, S, d, N)), S, d, N)
    allm = F.time_part_modes(d, N, n, tau, alpha, Yh, np.arange(m), c2=c2)
    assert np.abs(allm - full).max() <= 1e-12 * np.abs(full).max()
    sub = np.array([0, m // 3, m - 1])
    part = F.time_part_modes(d, N, n, tau, alpha, Yh[:, sub], sub, c2=c2)
    assert np.abs(part - full[:, sub]).max() <= 1e-12 * np.abs(full).max()
