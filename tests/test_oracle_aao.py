"""Pins of the oracle's all-at-once system and time stepping (Sec. 2,
Eqs. 1.2, 11-12, Lemma 2.3, Thm 2.1, Examples 1-2 of Sec. 4)."""
import numpy as np
import pytest

from oracle import aao, examples, fcd


def small_problem(M=7, Nt=8, alpha=1.5, kappa=1.0, seed=0):
    h = 1.0 / (M + 1)
    tau = 1.0 / Nt
    K = fcd.jacobian_1d(alpha, kappa, M, h)
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(M)
    f = rng.standard_normal((Nt, M))
    return K, tau, u0, f


def test_time_matrix_entries():
    C = aao.time_matrix_C(6)
    assert C[0, 0] == 1.0 and C[0, 1:].sum() == 0
    assert C[1, 0] == -2.0 and C[1, 1] == 1.5
    for k in range(2, 6):
        assert (C[k, k - 2], C[k, k - 1], C[k, k]) == (0.5, -2.0, 1.5)
    assert np.allclose(np.triu(C, 1), 0)


@pytest.mark.parametrize("Nt", [4, 8, 16, 40])
def test_lemma_2_3_norms(Nt):
    # Lemma 2.3 with the two labels exchanged: the max ROW sum of |C^{-1}| is Nt and the
    # max COLUMN sum is 3Nt/2 - 3/4 (1 - 3^{-Nt}) (the derivation in the proof sums the
    # last row for one and the first column for the other).
    Ci = np.linalg.inv(aao.time_matrix_C(Nt))
    assert abs(np.abs(Ci).sum(axis=1).max() - Nt) < 1e-9 * Nt
    assert abs(np.abs(Ci).sum(axis=0).max() - (1.5 * Nt - 0.75 * (1 - 3.0 ** -Nt))) < 1e-9 * Nt


@pytest.mark.parametrize("alpha,Nt,M", [(1.2, 8, 5), (1.5, 16, 7), (1.9, 12, 9)])
def test_theorem_2_1_singular_value_bounds(alpha, Nt, M):
    K, tau, _, _ = small_problem(M, Nt, alpha)
    A = aao.assemble_all_at_once(K, Nt, tau)
    s = np.linalg.svd(A, compute_uv=False)
    assert s.max() <= 4 + tau * np.linalg.norm(K, 2) + 1e-12
    assert s.min() >= np.sqrt(6) / (3 * Nt) - 1e-12


def test_matvec_equals_kronecker_assembly():
    K, tau, _, f = small_problem(9, 8)
    A = aao.assemble_all_at_once(K, 8, tau)
    np.testing.assert_allclose(aao.matvec(K, tau, f).ravel(), A @ f.ravel(), rtol=1e-13, atol=1e-13)


def test_matvec_rows_equal_matvec():
    M, Nt, alpha = 33, 16, 1.7
    K, tau, _, V = small_problem(M, Nt, alpha)
    c = tau * 1.0 / (1.0 / (M + 1)) ** alpha
    gs = c * fcd.fcd_weights(alpha, M)
    W = aao.matvec(K, tau, V)
    rows = [0, 1, 2, 7, 15, 15]
    cols = [0, 32, 5, 16, 0, 31]
    np.testing.assert_allclose(aao.matvec_rows(gs, V, rows, cols), W[rows, cols], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.9])
def test_sequential_bdf2_is_the_all_at_once_solution(alpha):
    K, tau, u0, f = small_problem(7, 8, alpha)
    F = aao.build_rhs(u0, f, tau)
    U = aao.sequential_bdf2(K, tau, u0, f)
    A = aao.assemble_all_at_once(K, 8, tau)
    np.testing.assert_allclose(U.ravel(), np.linalg.solve(A, F.ravel()), rtol=1e-12, atol=1e-12)
    assert aao.true_relative_residual(K, tau, F, U) < 1e-14


def test_scheme_equations_hold():
    # Eq. 1.2: (u^1 - u^0)/tau - K u^1 = f^1 and (3u^k - 4u^{k-1} + u^{k-2})/(2 tau) - K u^k = f^k
    K, tau, u0, f = small_problem(11, 10, 1.4)
    U = aao.sequential_bdf2(K, tau, u0, f)
    np.testing.assert_allclose((U[0] - u0) / tau - K @ U[0], f[0], rtol=1e-10, atol=1e-10)
    full = np.vstack([u0, U])
    for k in range(2, 11):
        lhs = (3 * full[k] - 4 * full[k - 1] + full[k - 2]) / (2 * tau) - K @ full[k]
        np.testing.assert_allclose(lhs, f[k - 1], rtol=1e-9, atol=1e-9)


def test_build_rhs_rows():
    u0 = np.arange(3.0)
    f = np.ones((4, 3))
    F = aao.build_rhs(u0, f, 0.5)
    np.testing.assert_array_equal(F[0], 0.5 + u0)
    np.testing.assert_array_equal(F[1], 0.5 - 0.5 * u0)
    np.testing.assert_array_equal(F[2:], 0.5)


def test_example1_err_columns(golden):
    # Tables 1-3: Err of the exactly solved system lies within the printed P_eps / P_1
    # values up to their 5-digit rounding and the GMRES tolerance (2e-4 relative).
    for a, Nt, N, e1, e2, _src in golden("ex1_err.txt"):
        e = examples.ex1_err(float(a), int(Nt), int(N))
        lo, hi = sorted((float(e1), float(e2)))
        dev = 0.0 if lo <= e <= hi else min(abs(e - lo), abs(e - hi)) / lo
        assert dev < 2e-4, (a, Nt, N, e, e1, e2)


def test_example2_err_columns(golden):
    for a1, a2, Nt, N, e1, e2, _src in golden("ex2_err.txt"):
        e = examples.ex2_err(float(a1), float(a2), int(Nt), int(N))
        lo, hi = sorted((float(e1), float(e2)))
        dev = 0.0 if lo <= e <= hi else min(abs(e - lo), abs(e - hi)) / lo
        assert dev < 2e-4, (a1, a2, Nt, N, e, e1, e2)


def test_second_order_in_tau_and_h():
    # Lemma 2.2 and the BDF2 scheme: refining tau and h together by 2 divides Err by ~4
    errs = [examples.ex1_err(1.5, n, n, kappa=1.0) for n in (32, 64, 128)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_2d_time_stepping_matches_dense_solve():
    ax, ay, Mx, My, Nt = 1.3, 1.7, 5, 4, 6
    hx, hy = 1 / (Mx + 1), 1 / (My + 1)
    tau = 1 / Nt
    Kx = fcd.jacobian_1d(ax, 1.0, Mx, hx)
    Ky = fcd.jacobian_1d(ay, 1.0, My, hy)
    K = fcd.jacobian_2d(ax, ay, 1.0, 1.0, Mx, My, hx, hy)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((My, Mx))
    f = rng.standard_normal((Nt, My, Mx))
    U = aao.sequential_bdf2_2d(Kx, Ky, tau, u0, f)
    F = aao.build_rhs(u0, f, tau)
    A = aao.assemble_all_at_once(K, Nt, tau)
    np.testing.assert_allclose(U.ravel(), np.linalg.solve(A, F.ravel()), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(aao.matvec_2d(Kx, Ky, tau, U).ravel(), A @ U.ravel(), rtol=1e-12, atol=1e-12)
