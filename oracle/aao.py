"""The all-at-once BDF2 system and its exact solution by time stepping.

Test infrastructure only (see :mod:`oracle`).

Layout: a space-time vector is a float64 array ``V[k, i]`` of shape
``(Nt, M)`` (row k = time level k+1, space contiguous), i.e. the paper's
stacking U = [u^1; u^2; ...; u^{Nt}] (Eq. 12).  2D vectors are
``V[k, j, i]`` with x (i) fastest.
"""
import numpy as np
import scipy.linalg as sla


def time_matrix_C(Nt):
    """The Nt x Nt BDF2 time matrix C of Eq. 1.7 (BDF1 in the first row)."""
    C = np.zeros((Nt, Nt))
    C[0, 0] = 1.0
    for k in range(1, Nt):
        C[k, k] = 1.5
        C[k, k - 1] = -2.0
        if k >= 2:
            C[k, k - 2] = 0.5
    return C


def build_rhs(u0, f, tau):
    """Right-hand side F of Eq. 12.

    F_1 = tau f^1 + u^0, F_2 = tau f^2 - u^0 / 2, F_k = tau f^k (k >= 3).
    ``f`` has shape (Nt, ...) holding f^1 .. f^Nt; ``u0`` has the shape of one
    time level.
    """
    F = tau * np.array(f, dtype=np.float64, copy=True)
    F[0] += u0
    if F.shape[0] > 1:
        F[1] -= 0.5 * u0
    return F


def assemble_all_at_once(K, Nt, tau):
    """Dense calA = C (x) I_s - tau I_t (x) K (Eq. 12).  Tiny sizes only."""
    Ms = K.shape[0]
    return np.kron(time_matrix_C(Nt), np.eye(Ms)) - tau * np.kron(np.eye(Nt), K)


def matvec(K, tau, V):
    """calA v = vec(V C^T) - tau vec(K V) (Sec. 3.2), in the row layout.

    Row k of the result is sum_j C[k, j] V[j] - tau K V[k].  The time part is
    a product with the dense C and the space part a product with the dense K
    (both library matmuls).
    """
    V = np.asarray(V, dtype=np.float64)
    Nt = V.shape[0]
    Vf = V.reshape(Nt, -1)
    W = time_matrix_C(Nt) @ Vf - tau * (Vf @ K.T)
    return W.reshape(V.shape)


def matvec_rows(g_scaled, V, rows, cols):
    """Selected entries of calA v (Eq. 12; the Toeplitz product of Sec. 3.2), each computed on its own.

    ``g_scaled[d]`` = c * g_d with c = tau*kappa/h^alpha, so that -tau K has
    entries g_scaled[|i-l|].  Returns W[rows[q], cols[q]] for every q:
    sum over the BDF band of C[k, k-j] V[k-j, i] plus sum_l c g_|i-l| V[k, l].
    For checking a full-size matvec at sampled outputs.
    """
    V = np.asarray(V, dtype=np.float64)
    Nt, M = V.shape
    out = np.empty(len(rows))
    for q, (k, i) in enumerate(zip(rows, cols)):
        if k == 0:
            band = V[0, i]
        elif k == 1:
            band = 1.5 * V[1, i] - 2.0 * V[0, i]
        else:
            band = 1.5 * V[k, i] - 2.0 * V[k - 1, i] + 0.5 * V[k - 2, i]
        d = np.abs(i - np.arange(M))
        out[q] = band + np.dot(g_scaled[d], V[k])
    return out


def matvec_2d(Kx, Ky, tau, V):
    """calA v for the 2D system (Eq. 12 with K of Eq. 4.2), K = I (x) Kx + Ky (x) I (x fastest).

    Row k: sum_j C[k, j] V[j] - tau (V[k] Kx^T + Ky V[k]) with V[k] of shape
    (My, Mx).  Library matmuls only.
    """
    V = np.asarray(V, dtype=np.float64)
    Nt = V.shape[0]
    C = time_matrix_C(Nt)
    W = np.einsum("kj,jyx->kyx", C, V)
    W -= tau * (np.einsum("kyx,ix->kyi", V, Kx) + np.einsum("jy,kyx->kjx", Ky, V))
    return W


def sequential_bdf2(K, tau, u0, f):
    """Solve calA U = F by time stepping with BDF1 then BDF2 (Eq. 1.2).

    (I - tau K) u^1 = tau f^1 + u^0
    (3/2 I - tau K) u^k = tau f^k + 2 u^{k-1} - u^{k-2} / 2   (k >= 2)
    Each matrix is LU-factorised once with partial pivoting (library routine)
    and the Nt steps are forward/back substitutions.  This is block forward
    substitution on the block lower-triangular calA, so it gives the unique
    solution of Eq. 12.  Returns U of shape (Nt, M).
    """
    M = K.shape[0]
    Nt = f.shape[0]
    I = np.eye(M)
    lu1 = sla.lu_factor(I - tau * K)
    lu2 = sla.lu_factor(1.5 * I - tau * K)
    U = np.empty((Nt, M))
    U[0] = sla.lu_solve(lu1, tau * f[0] + u0)
    prev2, prev1 = u0, U[0]
    for k in range(1, Nt):
        U[k] = sla.lu_solve(lu2, tau * f[k] + 2.0 * prev1 - 0.5 * prev2)
        prev2, prev1 = prev1, U[k]
    return U


def sequential_bdf2_2d(Kx, Ky, tau, u0, f):
    """2D time stepping (Eq. 1.2 with the Jacobian of Eq. 4.2), by fast
    diagonalisation.

    K = I (x) Kx + Ky (x) I (x fastest).  With Kx = Qx Lx Qx^T and
    Ky = Qy Ly Qy^T (symmetric eigendecompositions, library routine), a solve
    with (beta I - tau K) is: transform to the eigenbasis, divide by
    beta - tau (Lx[i] + Ly[j]), transform back.  ``u0`` has shape (My, Mx)
    and ``f`` shape (Nt, My, Mx).
    """
    Lx, Qx = np.linalg.eigh(Kx)
    Ly, Qy = np.linalg.eigh(Ky)
    lam = Ly[:, None] + Lx[None, :]

    def solve(beta, r):
        rt = Qy.T @ r @ Qx
        return Qy @ (rt / (beta - tau * lam)) @ Qx.T

    Nt = f.shape[0]
    U = np.empty_like(f, dtype=np.float64)
    U[0] = solve(1.0, tau * f[0] + u0)
    prev2, prev1 = u0, U[0]
    for k in range(1, Nt):
        U[k] = solve(1.5, tau * f[k] + 2.0 * prev1 - 0.5 * prev2)
        prev2, prev1 = prev1, U[k]
    return U


def windowed_bdf2(K, tau, u0, f, n_windows):
    """The windowed (restarted) scheme of Sec. 2.2 (the remark after Thm 2.1): [0, T_hat] is split into
    n_windows windows of Nt = f.shape[0] / n_windows steps each; window q is the all-at-once system of
    Eq. 12 with u^0 = the last snapshot of window q - 1 (u0 for q = 0), so every window starts again with
    the BDF1 step.  Each window is solved exactly by :func:`sequential_bdf2`.  ``f`` holds the sources of
    all n_windows * Nt levels; returns U of the same shape."""
    f = np.asarray(f, dtype=np.float64)
    Nt = f.shape[0] // n_windows
    assert Nt * n_windows == f.shape[0]
    U = np.empty_like(f)
    start = np.asarray(u0, dtype=np.float64)
    for q in range(n_windows):
        U[q * Nt:(q + 1) * Nt] = sequential_bdf2(K, tau, start, f[q * Nt:(q + 1) * Nt])
        start = U[(q + 1) * Nt - 1]
    return U


def true_relative_residual(K, tau, F, U):
    """TRR = ||F - calA U||_2 / ||F||_2 (Sec. 4), with the dense matvec."""
    R = F - matvec(K, tau, U)
    return np.linalg.norm(R.ravel()) / np.linalg.norm(np.asarray(F).ravel())
