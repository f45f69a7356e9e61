"""Manufactured-solution problems of Sec. 4 (Examples 1 and 2).

Test infrastructure only (see :mod:`oracle`).  Used to pin the oracle's
Jacobian, right-hand side and time stepping against the Err columns the
paper prints (Tables 1-6).
"""
import math
import numpy as np

from . import aao, fcd


def ex1_exact(alpha, x, t):
    """u(x, t) = 15 (1 + alpha/4) e^t x^3 (1-x)^3 (Example 1)."""
    return 15.0 * (1.0 + alpha / 4.0) * math.exp(t) * x ** 3 * (1.0 - x) ** 3


def ex1_source(alpha, kappa, x, t):
    """The source term f(x, t) printed for Example 1.

    u_t minus kappa times the Riesz derivative of u, with the Riesz derivative
    of x^3(1-x)^3 = x^3 - 3x^4 + 3x^5 - x^6 taken term by term from the
    Riemann-Liouville derivatives of powers of x and of (1-x).
    """
    c = 15.0 * (1.0 + alpha / 4.0) * math.exp(t)
    G = math.gamma
    br = (G(4) / G(4 - alpha) * (x ** (3 - alpha) + (1 - x) ** (3 - alpha))
          - 3 * G(5) / G(5 - alpha) * (x ** (4 - alpha) + (1 - x) ** (4 - alpha))
          + 3 * G(6) / G(6 - alpha) * (x ** (5 - alpha) + (1 - x) ** (5 - alpha))
          - G(7) / G(7 - alpha) * (x ** (6 - alpha) + (1 - x) ** (6 - alpha)))
    return c * x ** 3 * (1 - x) ** 3 + c * kappa / (2.0 * math.cos(alpha * math.pi / 2.0)) * br


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


_Q = {5: 16.0, 6: -32.0, 7: 24.0, 8: -8.0, 9: 1.0}


def _phi1(z):
    return z ** 4 * (2.0 - z) ** 4


def _riesz_part(alpha, z):
    """sum_{l=5}^{9} q_l Gamma(l) [z^{l-1-alpha} + (2-z)^{l-1-alpha}] / Gamma(l-alpha)."""
    G = math.gamma
    return sum(q * G(l) * (z ** (l - 1 - alpha) + (2.0 - z) ** (l - 1 - alpha)) / G(l - alpha)
               for l, q in _Q.items())


def ex2_exact(x, y, t):
    """u(x, y, t) = e^{-t/3} x^4 (2-x)^4 y^4 (2-y)^4 (Example 2)."""
    return math.exp(-t / 3.0) * _phi1(x) * _phi1(y)


def ex2_source(a1, a2, k1, k2, x, y, t):
    """Source term of Example 2 with the second sum taken in y (the printed
    formula repeats x there; the manufactured solution requires y)."""
    e = math.exp(-t / 3.0)
    return (-e / 3.0 * _phi1(x) * _phi1(y)
            + k1 * e / (2.0 * math.cos(a1 * math.pi / 2.0)) * _phi1(y) * _riesz_part(a1, x)
            + k2 * e / (2.0 * math.cos(a2 * math.pi / 2.0)) * _phi1(x) * _riesz_part(a2, y))


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
