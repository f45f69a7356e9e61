"""Pins of the oracle's restarted flexible GMRES (Sec. 4) against the exact
solution by time stepping and against the rank bound of Thm 3.1."""
import numpy as np
import pytest

from oracle import aao, fcd, gmres, precond


def problem(M, Nt, alpha, kappa=1.0, seed=0):
    h = 1.0 / (M + 1)
    tau = 1.0 / Nt
    K = fcd.jacobian_1d(alpha, kappa, M, h)
    rng = np.random.default_rng(seed)
    u0 = np.sin(np.pi * h * np.arange(1, M + 1))
    f = rng.uniform(-1, 1, (Nt, M))
    return K, tau, u0, f


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_preconditioned_fgmres_reaches_time_stepping_solution(alpha):
    M, Nt = 15, 16
    K, tau, u0, f = problem(M, Nt, alpha)
    F = aao.build_rhs(u0, f, tau)
    eps = precond.default_eps(tau)
    U, info = gmres.fgmres(lambda v: aao.matvec(K, tau, v),
                           lambda v: precond.precond_apply(K, tau, eps, v)[0], F, tol=1e-12)
    Useq = aao.sequential_bdf2(K, tau, u0, f)
    assert info["trr"] <= 1e-12
    assert np.linalg.norm(U - Useq) <= 1e-10 * np.linalg.norm(Useq)
    # Thm 3.1 (with rank 2M): GMRES on I + L needs at most 2M + 1 steps
    assert info["iters"] <= 2 * M + 1


def test_unpreconditioned_fgmres_also_converges():
    M, Nt = 7, 8
    K, tau, u0, f = problem(M, Nt, 1.5)
    F = aao.build_rhs(u0, f, tau)
    U, info = gmres.fgmres(lambda v: aao.matvec(K, tau, v), lambda v: v, F, tol=1e-12, restart=60)
    np.testing.assert_allclose(U, aao.sequential_bdf2(K, tau, u0, f), rtol=1e-9, atol=1e-10)


def test_p_eps_beats_p_1_at_small_kappa():
    # Tables 1-3 / Remark 3.2: with kappa = 0.01 the eps-circulant needs fewer iterations than P_1
    M, Nt, alpha = 31, 64, 1.5
    K, tau, u0, f = problem(M, Nt, alpha, kappa=0.01)
    F = aao.build_rhs(u0, f, tau)
    A = lambda v: aao.matvec(K, tau, v)
    _, ie = gmres.fgmres(A, lambda v: precond.precond_apply(K, tau, precond.default_eps(tau), v)[0], F, tol=1e-9)
    _, i1 = gmres.fgmres(A, lambda v: precond.precond_apply(K, tau, 1.0, v)[0], F, tol=1e-9)
    assert ie["iters"] < i1["iters"], (ie, i1)
