"""Pins of the oracle's FCD weights and Toeplitz matrix against facts the
paper and the mathematics fix (Eq. 2.4, Lemma 2.1, Lemma 2.2, Sec. 2.1)."""
import math

import numpy as np
import pytest

from oracle import fcd

ALPHAS = [1.1, 1.2, 1.5, 1.8, 1.9]


@pytest.mark.parametrize("alpha", ALPHAS)
def test_closed_form_matches_gamma_ratio_recurrence(alpha):
    # Gamma(z+1) = z Gamma(z) gives g_{k+1}/g_k = (k - alpha/2)/(alpha/2 + k + 1): an
    # independent route to the same numbers.
    g = fcd.fcd_weights(alpha, 201)
    r = np.empty(201)
    r[0] = math.gamma(1 + alpha) / math.gamma(1 + alpha / 2) ** 2
    for k in range(200):
        r[k + 1] = r[k] * (k - alpha / 2) / (alpha / 2 + k + 1)
    np.testing.assert_allclose(g, r, rtol=1e-12, atol=0)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_small_k_with_math_gamma(alpha):
    # direct evaluation of Eq. 2.4 with math.gamma (handles negative non-integer arguments)
    g = fcd.fcd_weights(alpha, 12)
    for k in range(12):
        want = (-1) ** k * math.gamma(1 + alpha) / (math.gamma(1 + alpha / 2 - k) * math.gamma(1 + alpha / 2 + k))
        assert abs(g[k] - want) <= 1e-14 * abs(want)


def test_alpha_two_is_the_second_difference():
    # Lemma 2.2: at order 2 the operator is the classical second difference [-1, 2, -1]
    g = fcd.fcd_weights(2.0 - 1e-15, 6)
    np.testing.assert_allclose(g, [2.0, -1.0, 0, 0, 0, 0], atol=1e-13)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_lemma_2_1_signs_and_zero_sum(alpha):
    K = 200000
    g = fcd.fcd_weights(alpha, K + 1)
    assert g[0] > 0 and np.all(g[1:] < 0)
    # sum over Z vanishes: g_0 + 2 sum_{k=1}^{K} g_k equals twice the tail sum_{k>K}|g_k|, whose
    # leading term follows from g_k ~ -Gamma(1+alpha) sin(pi alpha/2) / pi * k^{-1-alpha}
    s = g[0] + 2.0 * g[1:].sum()
    tail = 2.0 * math.gamma(1 + alpha) * math.sin(math.pi * alpha / 2) / (math.pi * alpha) * K ** (-alpha)
    assert s > 0
    assert abs(s - tail) <= 0.01 * tail


@pytest.mark.parametrize("alpha", ALPHAS)
def test_generating_function(alpha):
    # sum_k g_k e^{ik theta} = |2 sin(theta/2)|^alpha (symbol of the fractional centred difference)
    K = 400000
    g = fcd.fcd_weights(alpha, K + 1)
    k = np.arange(1, K + 1)
    for theta in (0.5, 1.0, 2.0, math.pi):
        val = g[0] + 2.0 * np.dot(g[1:], np.cos(k * theta))
        assert abs(val - abs(2 * math.sin(theta / 2)) ** alpha) < 1e-6


@pytest.mark.parametrize("alpha", ALPHAS)
def test_toeplitz_spd(alpha):
    T = fcd.toeplitz_T(alpha, 64)
    assert np.array_equal(T, T.T)
    ev = np.linalg.eigvalsh(T)
    assert ev.min() > 0
    # spectrum inside the range of the symbol (0, 2^alpha]
    assert ev.max() <= 2 ** alpha * (1 + 1e-12)


def test_jacobian_2d_is_kronecker_sum():
    Kx = fcd.jacobian_1d(1.3, 1.0, 5, 1 / 6)
    Ky = fcd.jacobian_1d(1.7, 0.5, 4, 1 / 5)
    K = fcd.jacobian_2d(1.3, 1.7, 1.0, 0.5, 5, 4, 1 / 6, 1 / 5)
    # acting on U[j, i] (x fastest): K vec(U) = vec(U Kx^T + Ky U)
    U = np.random.default_rng(0).standard_normal((4, 5))
    np.testing.assert_allclose(K @ U.ravel(), (U @ Kx.T + Ky @ U).ravel(), rtol=1e-13, atol=1e-13)


def test_alpha_two_is_the_classical_second_difference():
    """Lemma 2.2 at alpha = 2: the weights are [2, -1, 0, ...] exactly (1/Gamma vanishes at its poles)."""
    g = fcd.fcd_weights(2.0, 64)
    assert g[0] == 2.0 and g[1] == -1.0 and np.all(g[2:] == 0.0)
