"""Manufactured-solution problems of Sec. 4 (Examples 1 and 2).

Test infrastructure only (see :mod:`oracle`).  Used to pin the oracle's
Jacobian, right-hand side and time stepping against the Err columns the
paper prints (Tables 1-6).  The manufactured solutions and sources
themselves are problem data, shared with the bench through
``paper_2003_07020_gb300.workloads`` (the input module both sides use).
"""
import math
import numpy as np

from paper_2003_07020_gb300.workloads import ex1_exact, ex1_source, ex2_exact, ex2_source  # noqa: F401 (data)

from . import aao, fcd


def ex1_inputs(alpha, Nt, N, kappa=0.01, T=1.0, t0=0.0):
    """Example 1 on (0,1) with h = 1/N, M = N-1 interior points, tau = T/Nt: returns
    (x, K, u0, f) with u0 = u(x, t0) and f[k] = f(x, t0 + (k+1) tau), k < Nt."""
    h = 1.0 / N
    M = N - 1
    tau = T / Nt
    x = h * np.arange(1, M + 1)
    K = fcd.jacobian_1d(alpha, kappa, M, h)
    u0 = ex1_exact(alpha, x, t0)
    f = np.stack([ex1_source(alpha, kappa, x, t0 + (k + 1) * tau) for k in range(Nt)])
    return x, K, u0, f


def ex1_err(alpha, Nt, N, kappa=0.01, T=1.0):
    """Err = ||u* - u^{Nt}||_inf of Example 1 on (0,1) with h = 1/N, M = N-1
    interior points, tau = T/Nt, solved exactly by sequential BDF2."""
    x, K, u0, f = ex1_inputs(alpha, Nt, N, kappa, T)
    U = aao.sequential_bdf2(K, T / Nt, u0, f)
    return float(np.max(np.abs(ex1_exact(alpha, x, T) - U[-1])))


def ex2_inputs(a1, a2, Nt, N, kappa=0.01, T=2.0):
    """Example 2 on (0,2)^2 with N intervals per direction (mesh width 2/N, N-1 interior points
    each way), tau = T/Nt: returns (X, Y, Kx, Ky, u0, f), X[j, i] = x_i, Y[j, i] = y_j."""
    h = 2.0 / N
    M = N - 1
    tau = T / Nt
    z = h * np.arange(1, M + 1)
    X, Y = np.meshgrid(z, z)
    Kx = fcd.jacobian_1d(a1, kappa, M, h)
    Ky = fcd.jacobian_1d(a2, kappa, M, h)
    u0 = ex2_exact(X, Y, 0.0)
    f = np.stack([ex2_source(a1, a2, kappa, kappa, X, Y, (k + 1) * tau) for k in range(Nt)])
    return X, Y, Kx, Ky, u0, f


def ex2_err(a1, a2, Nt, N, kappa=0.01, T=2.0):
    """Err of Example 2 on (0,2)^2 with N intervals per direction (mesh width
    2/N, N-1 interior points each way), tau = T/Nt, solved exactly by
    sequential BDF2 with fast diagonalisation."""
    X, Y, Kx, Ky, u0, f = ex2_inputs(a1, a2, Nt, N, kappa, T)
    U = aao.sequential_bdf2_2d(Kx, Ky, T / Nt, u0, f)
    return float(np.max(np.abs(ex2_exact(X, Y, T) - U[-1])))
