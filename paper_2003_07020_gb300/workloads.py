"""Seeded synthetic inputs and the manufactured problems of the paper, shared
by the tests, the bench and the oracle-based checks.

Holds none of the method's arithmetic: only the initial value u^0 on the
mesh and the source samples f^1..f^Nt (and, for the paper's Examples 1 and 2,
their exact solutions).  Recipes (one per workload):

* ``"sine1_uniform"``: u^0(x) = sin(pi x); f i.i.d. uniform on [-1, 1].
* ``"sine8_normal"``:  u^0(x) = sum_{k=1}^{8} a_k sin(k pi x), a_k ~ N(0, 1);
  f i.i.d. N(0, 1).

The mesh is x_i = i h, h = 1/(M+1), i = 1..M (interior points of (0, 1)).
Random numbers come from numpy's PCG64 generator seeded with ``seed``; the
amplitudes a_k are drawn first, then f in row-major (Nt, M) order.
"""
import math

import numpy as np


def mesh(M):
    h = 1.0 / (M + 1)
    return h * np.arange(1, M + 1, dtype=np.float64)


def make_inputs(M, Nt, seed=0, recipe="sine8_normal"):
    """Returns (u0 [M], f [Nt, M]) as float64 numpy arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = mesh(M)
    if recipe == "sine1_uniform":
        u0 = np.sin(np.pi * x)
        f = rng.uniform(-1.0, 1.0, size=(Nt, M))
    elif recipe == "sine8_normal":
        a = rng.standard_normal(8)
        u0 = sum(a[k] * np.sin((k + 1) * np.pi * x) for k in range(8))
        f = rng.standard_normal((Nt, M))
    else:
        raise ValueError("unknown recipe %r" % recipe)
    return np.ascontiguousarray(u0), np.ascontiguousarray(f)


def make_inputs_2d(Mx, My, Nt, seed=0):
    """2D recipe "sine16_normal": u^0(x, y) = sum_{k,l=1}^{4} a_kl sin(k pi x) sin(l pi y), a_kl ~ N(0, 1)
    (16 modes, drawn first, row-major in (k, l)); f i.i.d. N(0, 1) of shape (Nt, My, Mx), x fastest.
    Returns (u0 [My, Mx], f [Nt, My, Mx])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((4, 4))
    x = mesh(Mx)
    y = mesh(My)
    sx = np.stack([np.sin((k + 1) * np.pi * x) for k in range(4)])
    sy = np.stack([np.sin((l + 1) * np.pi * y) for l in range(4)])
    u0 = np.einsum("kl,ly,kx->yx", a, sy, sx)
    f = rng.standard_normal((Nt, My, Mx))
    return np.ascontiguousarray(u0), np.ascontiguousarray(f)


def batched_instances(n=64, seed=0, Ms=(511, 1023, 2047, 4095), Nts=(128, 256, 512, 1024)):
    """Parameters of n independent 1D instances (the batched workload): M and Nt uniform over the given
    sets, alpha ~ U(1.1, 1.9), kappa ~ U(0.5, 2), inputs "sine8_normal" with seed 1000 + i.
    Returns a list of dicts (M, Nt, alpha, kappa, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = rng.choice(np.asarray(Ms), n)
    Nt = rng.choice(np.asarray(Nts), n)
    alpha = rng.uniform(1.1, 1.9, n)
    kappa = rng.uniform(0.5, 2.0, n)
    return [dict(M=int(M[i]), Nt=int(Nt[i]), alpha=float(alpha[i]), kappa=float(kappa[i]), seed=1000 + i)
            for i in range(n)]


def learned_instances(n, seed=0, M=1023, Nt=256, first_seed=0):
    """Parameters of n 1D instances of the learned warm-start workload: fixed M and Nt, alpha ~ U(1.1, 1.9),
    kappa = 1, inputs "sine8_normal" with seeds first_seed, first_seed + 1, ...  Training and held-out sets
    use disjoint seed ranges.  Returns a list of dicts (M, Nt, alpha, kappa, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    alpha = rng.uniform(1.1, 1.9, n)
    return [dict(M=int(M), Nt=int(Nt), alpha=float(alpha[i]), kappa=1.0, seed=first_seed + i) for i in range(n)]


def random_vector(Nt, M, seed=0):
    """A generic space-time vector with N(0, 1) entries (for operator tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((Nt, M))


# ---- the manufactured problems of Sec. 4 (Examples 1 and 2): data of the PDE, not of the method ----
def ex1_exact(alpha, x, t):
    """u(x, t) = 15 (1 + alpha/4) e^t x^3 (1-x)^3 (Example 1)."""
    return 15.0 * (1.0 + alpha / 4.0) * math.exp(t) * x ** 3 * (1.0 - x) ** 3


def ex1_source(alpha, kappa, x, t):
    """The source term f(x, t) printed for Example 1: u_t minus kappa times the Riesz derivative of u, the
    Riesz derivative of x^3(1-x)^3 = x^3 - 3x^4 + 3x^5 - x^6 taken term by term from the Riemann-Liouville
    derivatives of powers of x and of (1-x)."""
    c = 15.0 * (1.0 + alpha / 4.0) * math.exp(t)
    G = math.gamma
    br = (G(4) / G(4 - alpha) * (x ** (3 - alpha) + (1 - x) ** (3 - alpha))
          - 3 * G(5) / G(5 - alpha) * (x ** (4 - alpha) + (1 - x) ** (4 - alpha))
          + 3 * G(6) / G(6 - alpha) * (x ** (5 - alpha) + (1 - x) ** (5 - alpha))
          - G(7) / G(7 - alpha) * (x ** (6 - alpha) + (1 - x) ** (6 - alpha)))
    return c * x ** 3 * (1 - x) ** 3 + c * kappa / (2.0 * math.cos(alpha * math.pi / 2.0)) * br


def ex1_problem(alpha, Nt, N, kappa=0.01, T=1.0, t0=0.0):
    """Example 1 on (0,1) with h = 1/N, M = N - 1 interior points, tau = T/Nt: returns (x, u0, f) with
    u0 = u(x, t0) and f[k] = f(x, t0 + (k+1) tau), k < Nt."""
    h = 1.0 / N
    x = h * np.arange(1, N, dtype=np.float64)
    tau = T / Nt
    u0 = ex1_exact(alpha, x, t0)
    f = np.stack([ex1_source(alpha, kappa, x, t0 + (k + 1) * tau) for k in range(Nt)])
    return x, np.ascontiguousarray(u0), np.ascontiguousarray(f)


_Q2 = {5: 16.0, 6: -32.0, 7: 24.0, 8: -8.0, 9: 1.0}


def _phi2(z):
    return z ** 4 * (2.0 - z) ** 4


def _riesz_part2(alpha, z):
    """sum_{l=5}^{9} q_l Gamma(l) [z^{l-1-alpha} + (2-z)^{l-1-alpha}] / Gamma(l-alpha)."""
    G = math.gamma
    return sum(q * G(l) * (z ** (l - 1 - alpha) + (2.0 - z) ** (l - 1 - alpha)) / G(l - alpha)
               for l, q in _Q2.items())


def ex2_exact(x, y, t):
    """u(x, y, t) = e^{-t/3} x^4 (2-x)^4 y^4 (2-y)^4 (Example 2)."""
    return math.exp(-t / 3.0) * _phi2(x) * _phi2(y)


def ex2_source(a1, a2, k1, k2, x, y, t):
    """Source term of Example 2 with the second sum taken in y (the printed formula repeats x there; the
    manufactured solution requires y)."""
    e = math.exp(-t / 3.0)
    return (-e / 3.0 * _phi2(x) * _phi2(y)
            + k1 * e / (2.0 * math.cos(a1 * math.pi / 2.0)) * _phi2(y) * _riesz_part2(a1, x)
            + k2 * e / (2.0 * math.cos(a2 * math.pi / 2.0)) * _phi2(x) * _riesz_part2(a2, y))


def ex2_problem(a1, a2, Nt, N, kappa=0.01, T=2.0):
    """Example 2 on (0,2)^2 with N intervals per direction (mesh width 2/N, N - 1 interior points each way),
    tau = T/Nt: returns (X, Y, u0, f) with X[j, i] = x_i, Y[j, i] = y_j, f of shape (Nt, N-1, N-1)."""
    h = 2.0 / N
    z = h * np.arange(1, N, dtype=np.float64)
    X, Y = np.meshgrid(z, z)
    tau = T / Nt
    u0 = ex2_exact(X, Y, 0.0)
    # the source separates as e^{-t/3} times a fixed field
    base = ex2_source(a1, a2, kappa, kappa, X, Y, 0.0)
    f = np.empty((Nt,) + X.shape)
    for k in range(Nt):
        f[k] = math.exp(-(k + 1) * tau / 3.0) * base
    return X, Y, np.ascontiguousarray(u0), f
