"""Pins of the oracle FNO (the learned warm start of the shifted solves):
backward against central finite differences, and the full-mode spectral
layer with R = I reproducing its input."""
import numpy as np

from oracle import fno


def test_backward_matches_finite_differences():
    C, K, L, M = 4, 3, 2, 11
    rng = np.random.default_rng(0)
    theta = fno.init_params(1, C, K, L) + 0.05 * rng.standard_normal(fno.num_params(C, K, L))
    b = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    f = fno.features(b, 0.3 + 0.2j, 1.4)
    t = rng.standard_normal((M, 2))
    y, cache = fno.forward(theta, f, C, K, L)
    _, dy = fno.loss_and_dy(y, t)
    g = fno.backward(theta, cache, dy, C, K, L)
    h = 1e-6
    for j in rng.choice(theta.size, 60, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        lp, _ = fno.loss_and_dy(fno.forward(tp, f, C, K, L)[0], t)
        lm, _ = fno.loss_and_dy(fno.forward(tm, f, C, K, L)[0], t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, g[j])


def test_full_mode_identity_layer_returns_input():
    # with K = M//2 + 1 modes and R = I the spectral part is the inverse of the truncated DFT
    C, L, M = 3, 1, 9
    K = M // 2 + 1
    p = fno.unpack(np.zeros(fno.num_params(C, K, L)), C, K, L)
    p["lift_W"][:] = np.eye(C, 6)
    for k in range(K):
        p["R0"][k, :, :, 0] = np.eye(C)
    theta = np.concatenate([p[n].ravel() for n, _ in fno.layout(C, K, L)])
    b = np.random.default_rng(1).standard_normal(M) + 0j
    f = fno.features(b, 0.1 + 0.1j, 1.5)
    _, cache = fno.forward(theta, f, C, K, L)
    h0 = cache["hs"][0]
    # the last layer has no activation; z = s + 0 = h0 for odd M (no Nyquist mode)
    np.testing.assert_allclose(cache["zs"][0], h0, atol=1e-12)
