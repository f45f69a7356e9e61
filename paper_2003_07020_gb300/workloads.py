"""Seeded synthetic inputs for the 1D problem, shared by the tests, the
bench and the oracle-based checks.

Holds none of the method's arithmetic: only the initial value u^0 on the
mesh and the source samples f^1..f^Nt.  Recipes (one per workload):

* ``"sine1_uniform"``: u^0(x) = sin(pi x); f i.i.d. uniform on [-1, 1].
* ``"sine8_normal"``:  u^0(x) = sum_{k=1}^{8} a_k sin(k pi x), a_k ~ N(0, 1);
  f i.i.d. N(0, 1).

The mesh is x_i = i h, h = 1/(M+1), i = 1..M (interior points of (0, 1)).
Random numbers come from numpy's PCG64 generator seeded with ``seed``; the
amplitudes a_k are drawn first, then f in row-major (Nt, M) order.
"""
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
