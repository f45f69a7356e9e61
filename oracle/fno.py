"""Fourier neural operator for warm-starting the shifted solves of Step (b),
plain numpy FP64 forward and backward.

Test infrastructure only (see :mod:`oracle`).  The paper has no learned
component; this follows the architecture the GPU path implements (the
learned warm start), written out step by step:

  features f_i = [Re bh_i, Im bh_i, Re lambda, Im lambda, alpha, x_i],
                 bh = b / ||b||, x_i = (i+1)/(M+1)
  h0 = W_lift f + b_lift                               (6 -> C channels)
  for each Fourier layer l:
      H_k = sum_i h_i exp(-2 pi i i k / M),  k < K     (truncated DFT)
      G_k = R_l[k] H_k                                 (complex C x C per mode)
      s_i = (1/M) Re sum_{k<K} c_k G_k exp(+2 pi i i k / M),  c_0 = 1, c_k = 2
      z_i = s_i + W_l h_i + b_l
      h   = GELU(z) for all but the last layer, h = z for the last
  y_i = W_proj h_i + b_proj                            (C -> 2)
  x0  = ||b|| (y_0 + i y_1)

Loss of a sample with target t = x / ||b||: sum |y - t|^2 / sum |t|^2, averaged
over the batch.  Parameters live in one flat vector in the order
lift_W (C x 6), lift_b (C), then per layer R (K x C x C complex, re/im
interleaved), W (C x C), b (C), then proj_W (2 x C), proj_b (2).

Parity status: pinned by central finite differences of the loss (backward)
and by the identity that a spectral layer with all K = M//2 + 1 modes and
R = I returns its input (forward).
"""
import math

import numpy as np
from scipy.special import erf


def layout(C=32, K=16, L=4):
    """(name, shape) of every parameter block in flat order."""
    out = [("lift_W", (C, 6)), ("lift_b", (C,))]
    for l in range(L):
        out += [("R%d" % l, (K, C, C, 2)), ("W%d" % l, (C, C)), ("b%d" % l, (C,))]
    out += [("proj_W", (2, C)), ("proj_b", (2,))]
    return out


def unpack(theta, C=32, K=16, L=4):
    p, o = {}, 0
    for name, shape in layout(C, K, L):
        n = int(np.prod(shape))
        p[name] = theta[o:o + n].reshape(shape)
        o += n
    assert o == theta.size
    return p


def num_params(C=32, K=16, L=4):
    return sum(int(np.prod(s)) for _, s in layout(C, K, L))


def features(b, lam, alpha):
    """[M, 6] input features of one shifted system with right-hand side b."""
    M = b.size
    bh = b / np.linalg.norm(b)
    x = (np.arange(M) + 1.0) / (M + 1.0)
    f = np.empty((M, 6))
    f[:, 0], f[:, 1] = bh.real, bh.imag
    f[:, 2], f[:, 3] = lam.real, lam.imag
    f[:, 4] = alpha
    f[:, 5] = x
    return f


def _gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def _gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _modes(M, K):
    i = np.arange(M)[:, None]
    k = np.arange(K)[None, :]
    E = np.exp(-2j * np.pi * i * k / M)             # [M, K]
    c = np.where(np.arange(K) == 0, 1.0, 2.0)
    return E, c


def forward(theta, f, C=32, K=16, L=4):
    """y [M, 2] and the cache for backward."""
    p = unpack(theta, C, K, L)
    M = f.shape[0]
    E, c = _modes(M, K)
    h = f @ p["lift_W"].T + p["lift_b"]
    cache = {"f": f, "hs": [h], "zs": [], "Hs": []}
    for l in range(L):
        R = p["R%d" % l][..., 0] + 1j * p["R%d" % l][..., 1]      # [K, Cout, Cin]
        H = E.T @ h                                               # [K, C]
        G = np.einsum("koi,ki->ko", R, H)
        s = ((E.conj() * c[None, :]) @ G).real / M                # [M, C]
        z = s + h @ p["W%d" % l].T + p["b%d" % l]
        h = _gelu(z) if l < L - 1 else z
        cache["Hs"].append(H)
        cache["zs"].append(z)
        cache["hs"].append(h)
    y = h @ p["proj_W"].T + p["proj_b"]
    return y, cache


def loss_and_dy(y, t):
    """Per-sample loss sum |y - t|^2 / sum |t|^2 and its gradient in y; t as [M, 2]."""
    den = np.sum(t * t)
    e = y - t
    return float(np.sum(e * e) / den), 2.0 * e / den


def backward(theta, cache, dy, C=32, K=16, L=4):
    """Gradient of the loss in the flat parameter order."""
    p = unpack(theta, C, K, L)
    g = {name: np.zeros(shape) for name, shape in layout(C, K, L)}
    f = cache["f"]
    M = f.shape[0]
    E, c = _modes(M, K)
    hL = cache["hs"][L]
    g["proj_W"] = dy.T @ hL
    g["proj_b"] = dy.sum(0)
    dh = dy @ p["proj_W"]
    for l in range(L - 1, -1, -1):
        z = cache["zs"][l]
        dz = dh * _gelu_grad(z) if l < L - 1 else dh
        hp = cache["hs"][l]
        g["W%d" % l] = dz.T @ hp
        g["b%d" % l] = dz.sum(0)
        dhp = dz @ p["W%d" % l]
        # s = (1/M) Re(Ec G): complex gradient of G_k is (c_k / M) sum_i dz_i E_ik
        gG = (E * c[None, :]).T @ dz / M                            # [K, C]
        R = p["R%d" % l][..., 0] + 1j * p["R%d" % l][..., 1]
        H = cache["Hs"][l]
        gR = np.einsum("ko,ki->koi", gG, H.conj())
        g["R%d" % l] = np.stack([gR.real, gR.imag], axis=-1)
        gH = np.einsum("koi,ko->ki", R.conj(), gG)
        dhp += (E.conj() @ gH).real                                 # dL/dh_i = sum_k Re(gH_k e^{+i theta})
        dh = dhp
    g["lift_W"] = dh.T @ f
    g["lift_b"] = dh.sum(0)
    return np.concatenate([g[name].ravel() for name, _ in layout(C, K, L)])


def init_params(seed=0, C=32, K=16, L=4):
    """Scaled Gaussian initialisation (fan-in)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in layout(C, K, L):
        if name.startswith("R"):
            parts.append(rng.standard_normal(shape).ravel() / (C * math.sqrt(2.0)))
        elif name.endswith("_b") or name.startswith("b"):
            parts.append(np.zeros(int(np.prod(shape))))
        else:
            parts.append(rng.standard_normal(shape).ravel() / math.sqrt(shape[-1]))
    return np.concatenate(parts)


def predict(theta, b, lam, alpha, C=32, K=16, L=4):
    """x0 = ||b|| (y_0 + i y_1) for one system."""
    y, _ = forward(theta, features(b, lam, alpha), C, K, L)
    return np.linalg.norm(b) * (y[:, 0] + 1j * y[:, 1])
