"""The eps-circulant (generalised block-circulant) preconditioner.

Test infrastructure only (see :mod:`oracle`).

Paper: Sec. 3.1 (Eq. 1.11, Eq. 1.6a/b, Eq. 1.7x, Steps (a)-(c), Prop. 3.1,
Thm 3.1) and Sec. 3.2 (half of the shifted systems).  This code names the
circulant parameter ``eps`` (the paper's alpha) because ``alpha`` is the
fractional order here.

Step-(b) inner solver: the paper solves the shifted systems directly with a
tau-matrix approximation; the preconditioned conjugate-gradient form used
here is COCG (conjugate orthogonal CG: the bilinear form x^T y without
conjugation), because lambda_n I - tau K is complex symmetric, not
Hermitian, for Im lambda_n != 0.  The preconditioner is the Strang
circulant of T.
"""
import numpy as np
import scipy.linalg as sla


def default_eps(tau):
    """eps = min{0.5, 0.5 tau}, the choice of Sec. 4."""
    return min(0.5, 0.5 * tau)


def C_eps(Nt, eps):
    """The eps-circulant C_eps of Eq. 1.11 (Strang type).

    C with the wrap-around entries eps/2 at (0, Nt-2), (1, Nt-1) and -2 eps at
    (0, Nt-1).  Needs Nt >= 3.
    """
    C = np.zeros((Nt, Nt))
    for k in range(Nt):
        C[k, k] = 1.5
        if k >= 1:
            C[k, k - 1] = -2.0
        if k >= 2:
            C[k, k - 2] = 0.5
    C[0, Nt - 1] = -2.0 * eps
    C[0, Nt - 2] = 0.5 * eps
    C[1, Nt - 1] = 0.5 * eps
    return C


def eigenvalues_C_eps(Nt, eps):
    """lambda_n = sum_{j=0}^{2} r_j eps^{j/Nt} theta^{n j}, n = 0 .. Nt-1
    (Eq. 1.6a, 0-based n), r = (3/2, -2, 1/2), theta = exp(2 pi i / Nt)."""
    n = np.arange(Nt)
    theta = np.exp(2j * np.pi / Nt)
    r = (1.5, -2.0, 0.5)
    return sum(r[j] * eps ** (j / Nt) * theta ** (n * j) for j in range(3))


def dft_matrix(Nt):
    """The unitary Fourier matrix F_{Nt} of Eq. 1.6b: F[n, k] = theta^{nk}/sqrt(Nt)."""
    n = np.arange(Nt)
    return np.exp(2j * np.pi * np.outer(n, n) / Nt) / np.sqrt(Nt)


def P_eps_dense(K, tau, Nt, eps):
    """P_eps = C_eps (x) I_s - tau I_t (x) K (Sec. 3.1).  Tiny sizes only."""
    Ms = K.shape[0]
    return np.kron(C_eps(Nt, eps), np.eye(Ms)) - tau * np.kron(np.eye(Nt), K)


def precond_apply(K, tau, eps, V):
    """z = P_eps^{-1} v exactly, by the three steps of Sec. 3.1.

    Step-(a): z1 = (F (x) I)(Lambda^{-1} (x) I) v, Lambda^{-1} = diag(eps^{k/Nt})
    Step-(b): (lambda_n I - tau K) z2_n = z1_n, every n (dense complex solves)
    Step-(c): z = (Lambda (x) I)(F^* (x) I) z2
    with F the unitary DFT matrix (a dense complex matmul).  ``V`` has shape
    (Nt, Ms) (2D: flatten space first); K is the dense spatial Jacobian.
    The result is real to rounding; its real part is returned.
    """
    V = np.asarray(V, dtype=np.float64)
    Nt = V.shape[0]
    Vf = V.reshape(Nt, -1)
    Ms = Vf.shape[1]
    F = dft_matrix(Nt)
    scale = eps ** (np.arange(Nt) / Nt)
    Z1 = F @ (scale[:, None] * Vf)
    lam = eigenvalues_C_eps(Nt, eps)
    Z2 = np.empty_like(Z1)
    for n in range(Nt):
        Z2[n] = np.linalg.solve(lam[n] * np.eye(Ms) - tau * K, Z1[n])
    Z = (1.0 / scale)[:, None] * (F.conj().T @ Z2)
    return Z.real.reshape(V.shape), Z1, Z2


def time_dft_half(V, eps):
    """Step-(a) (Sec. 3.1, Eq. 1.6a; the half spectrum of Sec. 3.2) in the unnormalised form used by the GPU path:
    zhat_n = sum_k eps^{k/Nt} theta^{n k} v_k for n = 0 .. Nt/2.

    Equals sqrt(Nt) z1_n of :func:`precond_apply` (a dense complex matmul with
    the Vandermonde matrix theta^{nk}).
    """
    V = np.asarray(V, dtype=np.float64)
    Nt = V.shape[0]
    Vf = V.reshape(Nt, -1)
    n = np.arange(Nt // 2 + 1)
    k = np.arange(Nt)
    W = np.exp(2j * np.pi * np.outer(n, k) / Nt) * (eps ** (k / Nt))[None, :]
    return W @ Vf


def time_idft_half(X, eps, Nt):
    """Step-(c) from the half spectrum: z_k = eps^{-k/Nt} (1/Nt)
    sum_{n=0}^{Nt-1} x_n theta^{-n k} with x_{Nt-n} = conj(x_n) (Sec. 3.2).

    ``X`` holds x_0 .. x_{Nt/2} (Nt even).  The full spectrum is rebuilt by
    conjugate symmetry and the sum done as a dense complex matmul.
    """
    X = np.asarray(X)
    half = Nt // 2
    full = np.empty((Nt,) + X.shape[1:], dtype=np.complex128)
    full[: half + 1] = X
    for n in range(half + 1, Nt):
        full[n] = np.conj(X[Nt - n])
    n = np.arange(Nt)
    k = np.arange(Nt)
    W = np.exp(-2j * np.pi * np.outer(k, n) / Nt)
    Z = (W @ full.reshape(Nt, -1)) / Nt
    Z = Z.real * (eps ** (-k / Nt))[:, None]
    return Z.reshape((Nt,) + X.shape[1:])


def strang_symbol(g_scaled, M):
    """Step (b)'s circulant preconditioner (Sec. 3.1; the paper does not define a spatial Strang form, so
    the standard one is taken).  First column s of the Strang circulant of the symmetric Toeplitz matrix
    with first column g_scaled[0 .. M-1]: s_k = g_k for k <= M//2 and
    s_k = g_{M-k} otherwise.  Returns (s, eigenvalues), the eigenvalues being
    the DFT of s (real, since s is symmetric)."""
    k = np.arange(M)
    s = np.where(k <= M // 2, g_scaled[np.minimum(k, M - 1)], g_scaled[(M - k) % M])
    return s, np.fft.fft(s).real


def cocg(A, b, Pinv, tol, maxit, x0=None):
    """Preconditioned COCG for the complex symmetric system A x = b (a shifted system of Step (b), Sec. 3.1).

    Conjugate-orthogonal CG (van der Vorst and Melissen): preconditioned CG
    with the bilinear form (u, w) = u^T w instead of u^H w.  ``Pinv`` applies
    the (complex symmetric) preconditioner inverse.  Stops when
    ||r||_2 <= tol ||b||_2 or after ``maxit`` iterations (tol <= 0 runs exactly
    maxit iterations).  Returns (x, iterations, ||r||/||b||).
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    z = Pinv(r)
    p = z.copy()
    rho = r @ z
    it = 0
    res = np.linalg.norm(r) / nb
    while it < maxit and (tol <= 0 or res > tol):
        q = A @ p
        a = rho / (p @ q)
        x = x + a * p
        r = r - a * q
        it += 1
        res = np.linalg.norm(r) / nb
        if tol > 0 and res <= tol:
            break
        z = Pinv(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, it, res


def shifted_system(g_scaled, M, lam):
    """Dense lambda I + c T, with c T given by g_scaled (= -tau K): shifted system n of Step (b), Sec. 3.1."""
    idx = np.abs(np.arange(M)[:, None] - np.arange(M)[None, :])
    return lam * np.eye(M) + g_scaled[idx]


def strang_inverse(g_scaled, M, lam):
    """Step (b)'s preconditioner solve (Sec. 3.1): the map r -> (lambda I + c S)^{-1} r for the Strang circulant S,
    as a dense solve with the circulant matrix (library routine)."""
    s, _ = strang_symbol(g_scaled, M)
    P = lam * np.eye(M) + sla.circulant(s)
    lu = sla.lu_factor(P)
    return lambda r: sla.lu_solve(lu, r)


def tau_matrix(g_scaled, M):
    """The natural tau-algebra approximation tau(T) = T - H(T) of the
    symmetric Toeplitz T with first column g_scaled[0 .. M-1] (the tau-matrix
    approximation of Sec. 3.2 in the Bini-Di Benedetto form): H(T) is the
    Hankel matrix with first column (t_2, t_3, ..., t_{M-1}, 0, 0) and last
    column its reverse.  Dense; returns the M x M matrix."""
    idx = np.abs(np.arange(M)[:, None] - np.arange(M)[None, :])
    T = g_scaled[idx]
    t = np.zeros(2 * M + 2)
    t[:M] = g_scaled[:M]
    i = np.arange(M)[:, None]
    j = np.arange(M)[None, :]
    H = np.where(i + j + 2 <= M - 1, t[np.minimum(i + j + 2, 2 * M + 1)], 0.0)
    s = (M - 1 - i) + (M - 1 - j) + 2
    H = H + np.where(s <= M - 1, t[np.minimum(s, 2 * M + 1)], 0.0)
    return T - H


def dst1_matrix(M):
    """S_{jl} = sin(pi j l / (M+1)), j, l = 1..M (the DST-I matrix of Eq. 3.9
    without its normalisation)."""
    k = np.arange(1, M + 1)
    return np.sin(np.pi * np.outer(k, k) / (M + 1))


def tau_inverse(g_scaled, M, lam):
    """The map r -> (lambda I + tau(T))^{-1} r (the tau preconditioner of Sec. 3.2, Eq. 3.9) as a dense solve
    (library routine)."""
    P = lam * np.eye(M) + tau_matrix(g_scaled, M)
    lu = sla.lu_factor(P)
    return lambda r: sla.lu_solve(lu, r)


def jacobian_tau(alpha, kappa, M, h):
    """tau(A) = -(kappa / h^alpha) tau(T): the Jacobian with T replaced by its natural tau-matrix
    approximation (Sec. 3.2, Eq. 3.9; in 2D the Kronecker sum of two of these, Sec. 4 Ex. 2).  The paper's
    own Step (b) solves (lambda_n I - tau tau(A)) z_2 = z_1 directly (by DSTs); with this matrix in place
    of K, :func:`precond_apply` (1D) and :func:`precond_apply_2d` (2D) apply that preconditioner."""
    from . import fcd
    return -(kappa / h ** alpha) * tau_matrix(fcd.fcd_weights(alpha, M), M)


def time_S_eps(Nt, eps):
    """C_eps - C (Sec. 3.1, the remark on the polynomial preconditioner: S_eps = (C_eps - C) (x) I):
    nonzero only in time rows 0 and 1 (rank 2)."""
    from . import aao
    return C_eps(Nt, eps) - aao.time_matrix_C(Nt)


def P_eps_poly_apply(K, tau, eps, V, m, K_pre=None):
    """The m-step polynomial preconditioner of Sec. 3.1 (the remark after Thm 3.1):
    P_eps(m) v = sum_{k=0}^{m} (P_eps^{-1} S_eps)^k P_eps^{-1} v, S_eps = (C_eps - C) (x) I_s, a truncation
    of calA^{-1} = (I - P_eps^{-1} S_eps)^{-1} P_eps^{-1} since calA = P_eps - S_eps (the printed sum starts
    at k = 1; the truncation it defines starts at k = 0).  Evaluated by Horner's rule
    z <- P_eps^{-1} (v + S_eps z), m times after z = P_eps^{-1} v; P_eps^{-1} by :func:`precond_apply`
    (exact; with K_pre in place of K in Step (b) when given, e.g. :func:`jacobian_tau`)."""
    V = np.asarray(V, dtype=np.float64)
    Nt = V.shape[0]
    Kp = K if K_pre is None else K_pre
    S = time_S_eps(Nt, eps)
    z, _, _ = precond_apply(Kp, tau, eps, V)
    for _ in range(m):
        w = V.reshape(Nt, -1) + S @ z.reshape(Nt, -1)
        z, _, _ = precond_apply(Kp, tau, eps, w.reshape(V.shape))
    return z


def P_eps_matvec(K, tau, eps, Z):
    """P_eps z (Sec. 3.1, P_eps = C_eps (x) I - tau I (x) K) = vec(Z C_eps^T) - tau vec(K Z) in the row layout (dense C_eps and
    K; library matmuls).  For checking a computed z ~= P_eps^{-1} v by its
    residual at sizes where P_eps is too large to form."""
    Z = np.asarray(Z, dtype=np.float64)
    Nt = Z.shape[0]
    Zf = Z.reshape(Nt, -1)
    return (C_eps(Nt, eps) @ Zf - tau * (Zf @ K.T)).reshape(Z.shape)


def precond_apply_2d(Kx, Ky, tau, eps, V):
    """z = P_eps^{-1} v for the 2D system K = I (x) Kx + Ky (x) I (x fastest), by the
    three steps of Sec. 3.1 with Step (b) solved by fast diagonalisation:
    Kx = Qx Lx Qx^T, Ky = Qy Ly Qy^T (symmetric eigendecompositions, library
    routine), so (lambda_n I - tau K)^{-1} r = (Qy (x) Qx) [(Qy^T (x) Qx^T) r /
    (lambda_n - tau (Ly_j + Lx_i))].  ``V`` has shape (Nt, My, Mx)."""
    V = np.asarray(V, dtype=np.float64)
    Nt, My, Mx = V.shape
    F = dft_matrix(Nt)
    scale = eps ** (np.arange(Nt) / Nt)
    Z1 = F @ (scale[:, None] * V.reshape(Nt, -1))
    lam = eigenvalues_C_eps(Nt, eps)
    Lx, Qx = np.linalg.eigh(Kx)
    Ly, Qy = np.linalg.eigh(Ky)
    lam2 = Ly[:, None] + Lx[None, :]
    Z2 = np.empty_like(Z1)
    for n in range(Nt):
        rt = Qy.T @ Z1[n].reshape(My, Mx) @ Qx
        Z2[n] = (Qy @ (rt / (lam[n] - tau * lam2)) @ Qx.T).ravel()
    Z = (1.0 / scale)[:, None] * (F.conj().T @ Z2)
    return Z.real.reshape(V.shape)


def strang2d_inverse(gx_scaled, gy_scaled, Mx, My, lam):
    """Step (b)'s 2D preconditioner solve (Sec. 3.1, K of Eq. 4.2).  The map r -> (lambda I + I (x) S_x + S_y (x) I)^{-1} r for the 2D Strang (BCCB) preconditioner of the
    Kronecker-sum system (x fastest, r of shape (My, Mx)): S_x, S_y the Strang circulants of the scaled
    Toeplitz matrices with first columns gx_scaled, gy_scaled (:func:`strang_symbol`).  A BCCB matrix is
    diagonalised by the 2D DFT, so the solve divides the 2D DFT of r by lambda + eig_x[k] + eig_y[l] (library
    FFT routine)."""
    _, ex = strang_symbol(gx_scaled, Mx)
    _, ey = strang_symbol(gy_scaled, My)
    E = lam + ey[:, None] + ex[None, :]
    return lambda r: np.fft.ifft2(np.fft.fft2(np.asarray(r, dtype=np.complex128)) / E)


def P_eps_matvec_2d(Kx, Ky, tau, eps, Z):
    """P_eps z for the 2D system (Sec. 3.1 with K of Eq. 4.2): row k is sum_j C_eps[k, j] Z[j] - tau (Z[k] Kx^T +
    Ky Z[k])."""
    Z = np.asarray(Z, dtype=np.float64)
    Nt = Z.shape[0]
    W = np.einsum("kj,jyx->kyx", C_eps(Nt, eps), Z)
    W -= tau * (np.einsum("kyx,ix->kyi", Z, Kx) + np.einsum("jy,kyx->kjx", Ky, Z))
    return W
