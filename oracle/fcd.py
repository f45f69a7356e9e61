"""Fractional centred difference (FCD) weights and the Toeplitz Jacobian.

Test infrastructure only (see :mod:`oracle`).

Paper: Sec. 2.1, Eq. 2.3-2.4 (weights), Lemma 2.1 (their properties), the
matrix ``A = -kappa/h^gamma * T_x`` below Eq. 2.7 and, for 2D, Eq. 4.2.

Notation used in this code: ``alpha`` is the fractional order (the paper's
gamma); ``g[k]`` is the paper's omega_k.
"""
import numpy as np
from scipy.special import gammaln, gammasgn


def fcd_weights(alpha, n):
    """g_0 .. g_{n-1} from the closed form of Eq. 2.4.

    g_k = (-1)^k Gamma(1+alpha) / (Gamma(1+alpha/2-k) Gamma(1+alpha/2+k)),
    evaluated through log|Gamma| and the sign of Gamma (both library
    routines), so that it does not overflow for large k.  For 1 < alpha < 2
    none of the Gamma arguments is a pole; for alpha = 2 the argument
    1 + alpha/2 - k is a pole for every k >= 2, where 1/Gamma vanishes, so
    those weights are exactly 0 (the classical second difference [2, -1]).
    """
    k = np.arange(n, dtype=np.float64)
    a = float(alpha)
    arg = 1.0 + a / 2.0 - k
    pole = (arg <= 0) & (arg == np.floor(arg))
    with np.errstate(invalid="ignore"):
        lg = gammaln(1.0 + a) - gammaln(arg) - gammaln(1.0 + a / 2.0 + k)
        sgn = ((-1.0) ** k) * gammasgn(1.0 + a) * gammasgn(arg) * gammasgn(1.0 + a / 2.0 + k)
        g = sgn * np.exp(lg)
    return np.where(pole, 0.0, g)


def toeplitz_T(alpha, M):
    """The symmetric Toeplitz matrix T_x with entries omega_{i-j} (Sec. 2.1).

    Entry (i, j) is g_{|i-j|} since omega_{-l} = omega_l (Lemma 2.1).
    """
    g = fcd_weights(alpha, M)
    idx = np.abs(np.arange(M)[:, None] - np.arange(M)[None, :])
    return g[idx]


def jacobian_1d(alpha, kappa, M, h):
    """A = -(kappa / h^alpha) T_x, the M x M Jacobian (Sec. 2.1, matrix A).

    It is negative definite; this code calls it K.
    """
    return -(kappa / h ** alpha) * toeplitz_T(alpha, M)


def jacobian_2d(alpha_x, alpha_y, kappa_x, kappa_y, Mx, My, hx, hy):
    """2D Jacobian for unknowns ordered x fastest (index j*Mx + i).

    K = I_y (x) K_x + K_y (x) I_x, the Kronecker sum of Eq. 4.2 written for
    the x-fastest ordering.  Dense: small sizes only.
    """
    Kx = jacobian_1d(alpha_x, kappa_x, Mx, hx)
    Ky = jacobian_1d(alpha_y, kappa_y, My, hy)
    return np.kron(np.eye(My), Kx) + np.kron(Ky, np.eye(Mx))
