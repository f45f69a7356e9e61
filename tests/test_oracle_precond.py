"""Pins of the oracle's eps-circulant preconditioner (Sec. 3.1-3.2: Eq. 1.11,
Eq. 1.6a, Steps (a)-(c), Prop. 3.1, Thm 3.1, half of the systems) and of the
Step-(b) inner solver pieces (Strang circulant, natural tau matrix, COCG)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import aao, fcd, precond


def setup(M=7, Nt=8, alpha=1.5, kappa=1.0, seed=0):
    h = 1.0 / (M + 1)
    tau = 1.0 / Nt
    K = fcd.jacobian_1d(alpha, kappa, M, h)
    V = np.random.default_rng(seed).standard_normal((Nt, M))
    return K, tau, V


@pytest.mark.parametrize("Nt", [8, 16, 64])
@pytest.mark.parametrize("eps", [1.0, 0.5, 0.01, 1 / 128])
def test_eigenvalue_formula_matches_eig(Nt, eps):
    lam = precond.eigenvalues_C_eps(Nt, eps)
    ev = np.linalg.eigvals(precond.C_eps(Nt, eps))
    # match each formula eigenvalue to its nearest computed one
    d = np.abs(lam[:, None] - ev[None, :]).min(axis=1)
    assert d.max() < 1e-8
    # and the diagonalisation C_eps = V D V^{-1}, V = Lambda F^* (Eq. 1.6a)
    F = precond.dft_matrix(Nt)
    Lam = np.diag(eps ** (-np.arange(Nt) / Nt))
    Vm = Lam @ F.conj().T
    np.testing.assert_allclose(Vm @ np.diag(lam) @ np.linalg.inv(Vm), precond.C_eps(Nt, eps), atol=1e-10)


@pytest.mark.parametrize("Nt", [8, 64, 1024])
def test_proposition_3_1(Nt):
    for eps in (0.5, 1e-3, 0.5 / Nt):
        assert precond.eigenvalues_C_eps(Nt, eps).real.min() > 0
    lam1 = precond.eigenvalues_C_eps(Nt, 1.0)
    assert lam1.real.min() >= -1e-14 and abs(lam1[0]) < 1e-14


@pytest.mark.parametrize("alpha,eps", [(1.2, 0.5), (1.5, 1 / 16), (1.9, 1.0)])
def test_three_steps_equal_dense_inverse(alpha, eps):
    K, tau, V = setup(7, 8, alpha)
    z, _, _ = precond.precond_apply(K, tau, eps, V)
    want = np.linalg.solve(precond.P_eps_dense(K, tau, 8, eps), V.ravel())
    np.testing.assert_allclose(z.ravel(), want, rtol=1e-12, atol=1e-12)


def test_conjugate_symmetry_of_step_b():
    # Sec. 3.2: z2_{Nt-n} = conj(z2_n), so only n = 0 .. Nt/2 need solving
    K, tau, V = setup(9, 16, 1.7)
    _, Z1, Z2 = precond.precond_apply(K, tau, 1 / 32, V)
    for n in range(1, 16):
        np.testing.assert_allclose(Z1[16 - n], np.conj(Z1[n]), atol=1e-12)
        np.testing.assert_allclose(Z2[16 - n], np.conj(Z2[n]), atol=1e-12)


def test_half_spectrum_forms_reproduce_the_three_steps():
    Nt, M, eps, alpha = 16, 9, 1 / 32, 1.4
    K, tau, V = setup(M, Nt, alpha)
    z, Z1, Z2 = precond.precond_apply(K, tau, eps, V)
    zh = precond.time_dft_half(V, eps)
    np.testing.assert_allclose(zh, np.sqrt(Nt) * Z1[: Nt // 2 + 1], atol=1e-12)
    lam = precond.eigenvalues_C_eps(Nt, eps)
    xh = np.stack([np.linalg.solve(lam[n] * np.eye(M) - tau * K, zh[n]) for n in range(Nt // 2 + 1)])
    np.testing.assert_allclose(precond.time_idft_half(xh, eps, Nt), z, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("M,Nt", [(5, 8), (7, 16), (4, 12)])
def test_theorem_3_1_rank_is_2M(M, Nt):
    # P^{-1} calA - I = P^{-1}[(C - C_eps) (x) I]; rank(C - C_eps) = 2, so the rank is 2M
    # (the statement's "2 N_t" counts the wrong factor).
    K, tau, _ = setup(M, Nt, 1.5)
    A = aao.assemble_all_at_once(K, Nt, tau)
    P = precond.P_eps_dense(K, tau, Nt, 0.5)
    L = np.linalg.solve(P, A) - np.eye(M * Nt)
    s = np.linalg.svd(L, compute_uv=False)
    assert int((s > 1e-10 * s[0]).sum()) == 2 * M
    # eigenvalue clustering at 1 (Fig. 4.1): all but at most 2M eigenvalues equal 1
    ev = np.linalg.eigvals(np.linalg.solve(P, A))
    assert int((np.abs(ev - 1) > 1e-6).sum()) <= 2 * M


def test_strang_symbol_and_eigenvalues():
    M = 63
    g = fcd.fcd_weights(1.5, M)
    s, ev = precond.strang_symbol(g, M)
    C = sla.circulant(s)
    np.testing.assert_allclose(C, C.T, atol=0)
    np.testing.assert_allclose(np.sort(ev), np.linalg.eigvalsh(C), atol=1e-12)
    assert ev.min() > 0
    # the Strang circulant keeps the central band of T
    T = fcd.toeplitz_T(1.5, M)
    for d in range(M // 2 + 1):
        assert C[d, 0] == T[d, 0]


@pytest.mark.parametrize("M", [8, 15, 31])
def test_natural_tau_matrix_is_dst_diagonal(M):
    g = fcd.fcd_weights(1.3, M)
    Tt = precond.tau_matrix(g, M)
    S = precond.dst1_matrix(M)
    D = (2.0 / (M + 1)) * S @ Tt @ S
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-12
    # first column of tau(T) is (t0 - t2, t1 - t3, ..., t_{M-3} - t_{M-1}, t_{M-2}, t_{M-1})
    q = g[:M].copy()
    q[: M - 2] -= g[2:M]
    np.testing.assert_allclose(Tt[:, 0], q, atol=1e-15)
    # its eigenvalues follow from the first column: sigma_j = (S q)_j / sin(pi j/(M+1))
    j = np.arange(1, M + 1)
    np.testing.assert_allclose(np.diag(D), (S @ q) / np.sin(np.pi * j / (M + 1)), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("kind", ["strang", "tau"])
def test_cocg_solves_shifted_system(kind):
    M, Nt, alpha = 63, 64, 1.8
    c = (1.0 / Nt) / (1.0 / (M + 1)) ** alpha
    g = c * fcd.fcd_weights(alpha, M)
    lam = precond.eigenvalues_C_eps(Nt, 1 / 128)[3]
    A = precond.shifted_system(g, M, lam)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    Pinv = precond.strang_inverse(g, M, lam) if kind == "strang" else precond.tau_inverse(g, M, lam)
    x, it, res = precond.cocg(A, b, Pinv, 1e-12, 200)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-9)
    assert res <= 1e-12 and it < 40
    # with the exact inverse as preconditioner one iteration solves it
    lu = sla.lu_factor(A)
    x1, it1, _ = precond.cocg(A, b, lambda r: sla.lu_solve(lu, r), 0.0, 1)
    np.testing.assert_allclose(x1, np.linalg.solve(A, b), rtol=1e-10, atol=1e-10)
    # the shifted system is complex symmetric, not Hermitian
    assert np.allclose(A, A.T) and not np.allclose(A, A.conj().T)


def test_2d_three_steps_by_fast_diagonalisation_equal_dense():
    Mx, My, Nt, tau, eps = 5, 3, 8, 1 / 8, 1 / 16
    Kx = fcd.jacobian_1d(1.3, 1.0, Mx, 1 / (Mx + 1))
    Ky = fcd.jacobian_1d(1.7, 0.5, My, 1 / (My + 1))
    K = fcd.jacobian_2d(1.3, 1.7, 1.0, 0.5, Mx, My, 1 / (Mx + 1), 1 / (My + 1))
    V = np.random.default_rng(2).standard_normal((Nt, My, Mx))
    z = precond.precond_apply_2d(Kx, Ky, tau, eps, V)
    want = np.linalg.solve(precond.P_eps_dense(K, tau, Nt, eps), V.ravel())
    np.testing.assert_allclose(z.ravel(), want, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(precond.P_eps_matvec_2d(Kx, Ky, tau, eps, z).ravel(),
                               precond.P_eps_dense(K, tau, Nt, eps) @ z.ravel(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("M,Nt", [(5, 8), (9, 16), (4, 12)])
@pytest.mark.parametrize("eps", [1.0, 0.5, 1 / 16])
def test_P_eps_matvec_equals_the_assembled_preconditioner(M, Nt, eps):
    # P_eps = C_eps (x) I_s - tau I_t (x) K (Sec. 3.1) assembled by Kronecker products against the
    # row form of P_eps_matvec: a transposed C_eps or K, or a sign slip, fails here
    K, tau, _ = setup(M, Nt, 1.6)
    Z = np.random.default_rng(9).standard_normal((Nt, M))
    want = precond.P_eps_dense(K, tau, Nt, eps) @ Z.ravel()
    np.testing.assert_allclose(precond.P_eps_matvec(K, tau, eps, Z).ravel(), want, rtol=1e-13, atol=1e-13)
    # P_eps - calA = (C_eps - C) (x) I (Thm 3.1): only time rows 0 and 1 differ from the all-at-once
    # product, by (1/2) z_0 + (eps/2) z_{Nt-2} - 2 eps z_{Nt-1} and (eps/2) z_{Nt-1}
    D = precond.P_eps_matvec(K, tau, eps, Z) - aao.matvec(K, tau, Z)
    np.testing.assert_allclose(D[0], 0.5 * Z[0] + 0.5 * eps * Z[Nt - 2] - 2 * eps * Z[Nt - 1], atol=1e-13)
    np.testing.assert_allclose(D[1], 0.5 * eps * Z[Nt - 1], atol=1e-13)
    np.testing.assert_allclose(D[2:], 0.0, atol=1e-13)
    # and it inverts the three-step apply: P_eps (P_eps^{-1} v) = v
    z, _, _ = precond.precond_apply(K, tau, eps, Z)
    np.testing.assert_allclose(precond.P_eps_matvec(K, tau, eps, z), Z, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("Mx,My", [(7, 5), (15, 15), (9, 4)])
def test_strang2d_inverse_is_the_dense_circulant_sum_solve(Mx, My):
    # the BCCB Strang preconditioner I (x) S_x + S_y (x) I, assembled densely from scipy's circulant matrices
    gx = 40.0 * fcd.fcd_weights(1.3, Mx)
    gy = 25.0 * fcd.fcd_weights(1.8, My)
    lam = precond.eigenvalues_C_eps(16, 1 / 32)[3]
    sx, _ = precond.strang_symbol(gx, Mx)
    sy, _ = precond.strang_symbol(gy, My)
    P = lam * np.eye(Mx * My) + np.kron(np.eye(My), sla.circulant(sx)) + np.kron(sla.circulant(sy), np.eye(Mx))
    rng = np.random.default_rng(Mx * My)
    r = rng.standard_normal((My, Mx)) + 1j * rng.standard_normal((My, Mx))
    z = precond.strang2d_inverse(gx, gy, Mx, My, lam)(r)
    np.testing.assert_allclose(z.ravel(), np.linalg.solve(P, r.ravel()), rtol=1e-12, atol=1e-12)
    # and it keeps the central band of the 2D Toeplitz operator: for My = 1 it is the 1D Strang inverse
    z1 = precond.strang2d_inverse(gx, np.array([0.0]), Mx, 1, lam)(r[:1])
    np.testing.assert_allclose(z1.ravel(), precond.strang_inverse(gx, Mx, lam)(r[0]), rtol=1e-12, atol=1e-13)
