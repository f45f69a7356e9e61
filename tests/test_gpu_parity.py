"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.

Tolerances (stated per check below):
  * matvec (FP64 FFT, Sec. 3.2): relative 1e-13 in 2-norm at small sizes and
    1e-12 of the row scale at sampled full-size outputs (FFT rounding is
    about eps * log2(L) relative to c ||T|| ||v||);
  * preconditioner (Sec. 3.1): FP64 path with inner tol 1e-12 -> residual
    ||P z - v|| / ||v|| <= 1e-10 and z within 1e-9; mixed path with inner tol
    t = 1e-6 in FP32 -> ||z - z_exact|| / ||z_exact|| <= 4 (t + 64 u32) / eps:
    Step (c) multiplies time row k by eps^{-k/Nt}, so any relative error of
    the FP32 spectrum (inner tolerance plus FP32 rounding, u32 = 2^-24) is
    amplified up to cond(V_eps) = 1/eps (the conditioning of V_eps noted
    after Eq. 1.6b); and, system by system, the residual of every shifted
    system (lambda_n I - tau K) x_n = y_n recovered through exact FP64
    Steps (a)/(c) is at most t + 16 u32 ||A_n|| ||x_n|| / ||y_n||;
  * solve: true relative residual <= 1e-10 (computed by the oracle) and
    ||U - U_seq|| / ||U_seq|| <= 1e-10 (FP64 path) or 1e-9 (mixed path).
"""
import numpy as np
import pytest

from paper_2003_07020_gb300 import aao, workloads
from oracle import aao as oaao, fcd, precond as oprec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def jac(M, alpha, kappa=1.0):
    return fcd.jacobian_1d(alpha, kappa, M, 1.0 / (M + 1))


def mixed_eps(tau):
    """The library's default circulant parameter for the mixed path: max(min(0.5, 0.5 tau), 1/16)."""
    return max(min(0.5, 0.5 * tau), 1.0 / 16)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


# ---------------------------------------------------------------- matvec
@pytest.mark.parametrize("M,Nt,alpha", [(63, 64, 1.5), (100, 16, 1.2), (1, 4, 1.5), (2, 8, 1.9),
                                        (8, 4, 1.4), (16, 8, 1.7), (1023, 32, 1.8), (4095, 8, 1.3)])
@pytest.mark.parametrize("kind", [aao.AAO_MATVEC_NTT, aao.AAO_MATVEC_FFT64])
def test_matvec_matches_dense_oracle(M, Nt, alpha, kind):
    v = workloads.random_vector(Nt, M, seed=M + Nt)
    with aao.Plan(M, Nt, alpha, matvec=kind) as plan:
        w = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.matvec(cu(v), w)
        torch.cuda.synchronize()
    ref = oaao.matvec(jac(M, alpha), 1.0 / Nt, v)
    assert rel(host(w), ref) <= 1e-13


@pytest.mark.parametrize("kind", [aao.AAO_MATVEC_NTT, aao.AAO_MATVEC_FFT64])
def test_matvec_full_size_sampled(kind):
    M, Nt, alpha = 8191, 1024, 1.8
    v = workloads.random_vector(Nt, M, seed=7)
    with aao.Plan(M, Nt, alpha, matvec=kind) as plan:
        w = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.matvec(cu(v), w)
        torch.cuda.synchronize()
    W = host(w)
    c = (1.0 / Nt) / (1.0 / (M + 1)) ** alpha
    gs = c * fcd.fcd_weights(alpha, M)
    rng = np.random.default_rng(0)
    rows = np.r_[[0, 0, 1, 1, 2, Nt - 1, Nt - 1], rng.integers(0, Nt, 57)]
    cols = np.r_[[0, M - 1, 0, 4096, M - 1, 0, M - 1], rng.integers(0, M, 57)]
    ref = oaao.matvec_rows(gs, v, rows, cols)
    scale = np.abs(ref).max()
    assert np.abs(W[rows, cols] - ref).max() <= 1e-12 * scale


# ---------------------------------------------------------------- preconditioner
PREC_CASES = [(63, 64, 1.5), (100, 16, 1.2), (255, 32, 1.8), (1023, 16, 1.3), (3, 4, 1.5)]


@pytest.mark.parametrize("M,Nt,alpha", PREC_CASES)
@pytest.mark.parametrize("inner", [aao.AAO_INNER_STRANG, aao.AAO_INNER_TAU])
def test_precond_fp64_matches_three_step_oracle(M, Nt, alpha, inner):
    if inner == aao.AAO_INNER_TAU and (M + 1) & M:
        pytest.skip("tau preconditioner needs M+1 a power of two")
    v = workloads.random_vector(Nt, M, seed=3)
    tau = 1.0 / Nt
    eps = oprec.default_eps(tau)
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_FP64, inner=inner) as plan:
        z = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        torch.cuda.synchronize()
    K = jac(M, alpha)
    zr, _, _ = oprec.precond_apply(K, tau, eps, v)
    Z = host(z)
    assert rel(oprec.P_eps_matvec(K, tau, eps, Z), v) <= 1e-10
    assert rel(Z, zr) <= 1e-9


@pytest.mark.parametrize("M,Nt,alpha", PREC_CASES)
@pytest.mark.parametrize("inner", [aao.AAO_INNER_STRANG, aao.AAO_INNER_TAU])
def test_precond_mixed_residual(M, Nt, alpha, inner):
    if inner == aao.AAO_INNER_TAU and (M + 1) & M:
        pytest.skip("tau preconditioner needs M+1 a power of two")
    v = workloads.random_vector(Nt, M, seed=4)
    tau = 1.0 / Nt
    eps = mixed_eps(tau)
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED, inner=inner) as plan:
        z = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        torch.cuda.synchronize()
    K = jac(M, alpha)
    zr, _, _ = oprec.precond_apply(K, tau, eps, v)
    err = rel(host(z), zr)
    bound = 4 * (1e-6 + 64 * 2.0 ** -24) / eps
    assert err <= bound, (err, bound, rel(oprec.P_eps_matvec(K, tau, eps, host(z)), v))


@pytest.mark.parametrize("M,Nt,alpha", PREC_CASES + [(255, 128, 1.8), (511, 256, 1.5)])
@pytest.mark.parametrize("inner", [aao.AAO_INNER_STRANG, aao.AAO_INNER_TAU])
def test_precond_mixed_residual_of_every_shifted_system(M, Nt, alpha, inner):
    # Step (b) seen system by system.  Inverting the GPU's Step (c) exactly (in FP64: Step (a) of z is
    # the spectrum x_n that Step (c) received) and applying Step (a) exactly to v gives, for every
    # frequency n, the residual of the shifted system (lambda_n I - tau K) x_n = y_n (Sec. 3.1).  FP32
    # COCG stops at ||r|| <= t ||y_n|| on its recurrence residual, t = 1e-6; the true residual differs by
    # the FP32 rounding of the recurrence, modelled as gamma u32 kappa_n with kappa_n =
    # ||A_n|| ||x_n|| / ||y_n|| (A_n is normal: ||A_n|| = max_j |lambda_n - tau mu_j(K)|) and
    # gamma = 16, which covers a root-sum-square accumulation sqrt(k log2 L) of up to k = 18
    # iterations at L = 2^14.  A Step (b) defect of 1e-4 fails this on the well-conditioned systems.
    if inner == aao.AAO_INNER_TAU and (M + 1) & M:
        pytest.skip("tau preconditioner needs M+1 a power of two")
    v = workloads.random_vector(Nt, M, seed=4)
    tau = 1.0 / Nt
    eps = mixed_eps(tau)
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED, inner=inner) as plan:
        z = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        its, flags = plan.inner_record()
    assert (flags == 0).all(), flags
    K = jac(M, alpha)
    mu = np.linalg.eigvalsh(K)
    lam = oprec.eigenvalues_C_eps(Nt, eps)
    Y = oprec.time_dft_half(v, eps)
    X = oprec.time_dft_half(host(z), eps)
    u32, t, gamma = 2.0 ** -24, 1e-6, 16.0
    worst = 0.0
    for n in range(Nt // 2 + 1):
        A = lam[n] * np.eye(M) - tau * K
        ny = np.linalg.norm(Y[n])
        res = np.linalg.norm(Y[n] - A @ X[n]) / ny
        kappa = np.abs(lam[n] - tau * mu).max() * np.linalg.norm(X[n]) / ny
        bound = t + gamma * u32 * kappa
        worst = max(worst, res / bound)
        assert res <= bound, (n, res, bound, its[n])
    assert worst > 0.01, worst  # the check is not vacuous


def test_precond_aliasing_allowed():
    M, Nt = 63, 16
    v = workloads.random_vector(Nt, M, seed=5)
    with aao.Plan(M, Nt, 1.5, prec=aao.AAO_PREC_FP64) as plan:
        a = cu(v)
        b = torch.empty_like(a)
        plan.bc_precond_apply(a, b)
        plan.bc_precond_apply(a, a)
        torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_precond_full_size_mixed_residual():
    M, Nt, alpha = 8191, 1024, 1.8
    v = workloads.random_vector(Nt, M, seed=9)
    tau = 1.0 / Nt
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED) as plan:
        z = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        torch.cuda.synchronize()
    K = jac(M, alpha)
    # residual of the eps-circulant equation; the bound follows the z-error bound above
    # times ||P_eps|| ||z|| / ||v||, evaluated with ||P_eps|| <= 4 + c 2^alpha
    eps = mixed_eps(tau)
    Z = host(z)
    res = rel(oprec.P_eps_matvec(K, tau, eps, Z), v)
    c = tau / (1.0 / (M + 1)) ** alpha
    bound = 4 * (1e-6 + 64 * 2.0 ** -24) / eps * (4 + c * 2 ** alpha) * np.linalg.norm(Z) / np.linalg.norm(v)
    assert res <= bound, (res, bound)


# ---------------------------------------------------------------- right-hand side
def test_build_rhs():
    M, Nt = 37, 8
    u0, f = workloads.make_inputs(M, Nt, seed=1)
    with aao.Plan(M, Nt, 1.5) as plan:
        F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        torch.cuda.synchronize()
    np.testing.assert_allclose(host(F), oaao.build_rhs(u0, f, 1.0 / Nt), rtol=1e-15, atol=1e-15)


# ---------------------------------------------------------------- solve
def solve_case(M, Nt, alpha, prec, inner, recipe="sine8_normal", seed=0, matvec=aao.AAO_MATVEC_FFT64):
    u0, f = workloads.make_inputs(M, Nt, seed=seed, recipe=recipe)
    with aao.Plan(M, Nt, alpha, prec=prec, inner=inner, matvec=matvec) as plan:
        F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        U = torch.zeros_like(F)
        plan.build_rhs(cu(u0), cu(f), F)
        info = plan.gmres_solve(F, U)
    return u0, f, host(U), info


@pytest.mark.parametrize("prec,bound", [(aao.AAO_PREC_FP64, 1e-10), (aao.AAO_PREC_MIXED, 1e-9)])
@pytest.mark.parametrize("inner", [aao.AAO_INNER_STRANG, aao.AAO_INNER_TAU])
@pytest.mark.parametrize("M,Nt,alpha,recipe", [(63, 64, 1.5, "sine1_uniform"), (255, 128, 1.8, "sine8_normal"),
                                               (1023, 32, 1.2, "sine8_normal")])
def test_gmres_solve_matches_time_stepping(M, Nt, alpha, recipe, prec, bound, inner):
    u0, f, U, info = solve_case(M, Nt, alpha, prec, inner, recipe)
    K = jac(M, alpha)
    tau = 1.0 / Nt
    Useq = oaao.sequential_bdf2(K, tau, u0, f)
    trr = oaao.true_relative_residual(K, tau, oaao.build_rhs(u0, f, tau), U)
    assert info["true_rel_res"] <= 1e-10 and trr <= 1e-10, (info, trr)
    assert rel(U, Useq) <= bound, (rel(U, Useq), info)


@pytest.mark.parametrize("kind", [aao.AAO_MATVEC_FFT64, aao.AAO_MATVEC_NTT])
def test_gmres_full_size_config(kind):
    M, Nt, alpha = 8191, 1024, 1.8
    u0, f, U, info = solve_case(M, Nt, alpha, aao.AAO_PREC_MIXED, aao.AAO_INNER_STRANG, matvec=kind)
    K = jac(M, alpha)
    tau = 1.0 / Nt
    F = oaao.build_rhs(u0, f, tau)
    trr = oaao.true_relative_residual(K, tau, F, U)
    assert info["true_rel_res"] <= 1e-10 and trr <= 1e-10, (info, trr)
    Useq = oaao.sequential_bdf2(K, tau, u0, f)
    assert rel(U, Useq) <= 1e-9, rel(U, Useq)


def test_gmres_host_buffers_equal_device_path():
    M, Nt, alpha = 255, 64, 1.5
    u0, f = workloads.make_inputs(M, Nt, seed=2)
    F = oaao.build_rhs(u0, f, 1.0 / Nt)
    with aao.Plan(M, Nt, alpha) as plan:
        Uh = np.zeros((Nt, M))
        info_h = plan.gmres_solve_host(np.ascontiguousarray(F), Uh)
        Ud = torch.zeros((Nt, M), dtype=torch.float64, device=DEV)
        info_d = plan.gmres_solve(cu(F), Ud)
    assert info_h["outer_iters"] == info_d["outer_iters"]
    np.testing.assert_array_equal(Uh, host(Ud))


def test_zero_rhs_and_nonfinite_rhs():
    M, Nt = 31, 8
    with aao.Plan(M, Nt, 1.5) as plan:
        F = torch.zeros((Nt, M), dtype=torch.float64, device=DEV)
        U = torch.ones_like(F)
        info = plan.gmres_solve(F, U)
        assert info["outer_iters"] == 0 and torch.count_nonzero(U) == 0
        F[3, 4] = float("nan")
        with pytest.raises(aao.AaoError) as e:
            plan.gmres_solve(F, U)
        assert e.value.status == aao.AAO_ENONFINITE


def test_iteration_cap_reports_noconv():
    M, Nt = 63, 64
    u0, f = workloads.make_inputs(M, Nt, seed=0)
    with aao.Plan(M, Nt, 1.5, restart=1, max_cycles=1) as plan:
        F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        U = torch.zeros_like(F)
        with pytest.raises(aao.AaoError) as e:
            plan.gmres_solve(F, U)
        assert e.value.status == aao.AAO_ENOCONV


def test_ntt_matvec_edge_rows():
    """Exact-integer matvec: zero rows, rows of very different scale (per-row quantisation), a single
    huge entry, FP32 input (the Z basis), and a non-finite entry that must reach the output."""
    M, Nt, alpha = 255, 8, 1.7
    rng = np.random.default_rng(3)
    v = rng.standard_normal((Nt, M))
    v[1] = 0.0
    v[2] *= 1e-150
    v[3] *= 1e100
    v[4] = 0.0
    v[4, 17] = 3.0
    with aao.Plan(M, Nt, alpha, matvec=aao.AAO_MATVEC_NTT) as plan:
        w = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.matvec(cu(v), w)
        torch.cuda.synchronize()
        W = host(w)
        K = jac(M, alpha)
        ref = oaao.matvec(K, 1.0 / Nt, v)
        for k in range(Nt):  # row-wise relative accuracy (the time band mixes rows of different scale)
            nr = np.linalg.norm(ref[k])
            assert np.linalg.norm(W[k] - ref[k]) <= 1e-13 * nr + 1e-300, k
        vbad = v.copy()
        vbad[5, 3] = np.nan
        plan.matvec(cu(vbad), w)
        torch.cuda.synchronize()
        W = host(w)
        assert np.isnan(W[5]).all() and np.isfinite(W[:5]).all()


@pytest.mark.parametrize("alpha,kappa,T", [(2.0, 1.0, 1.0), (1.01, 1.0, 1.0), (1.5, 0.01, 2.0), (1.9, 3.0, 0.5)])
@pytest.mark.parametrize("prec", [aao.AAO_PREC_MIXED, aao.AAO_PREC_FP64])
def test_gmres_parameter_extremes(alpha, kappa, T, prec):
    """alpha = 2 (the classical Laplacian stencil [2, -1]: the quantised stencil tail is exactly zero), alpha near
    1, the small kappa of the paper's tables, and T != 1 (tau = T / Nt), against sequential BDF2."""
    M, Nt = 127, 32
    u0, f = workloads.make_inputs(M, Nt, seed=11)
    tau = T / Nt
    with aao.Plan(M, Nt, alpha, kappa=kappa, T=T, prec=prec) as plan:
        F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        U = torch.zeros_like(F)
        info = plan.gmres_solve(F, U)
    K = fcd.jacobian_1d(alpha, kappa, M, 1.0 / (M + 1))
    Fh = oaao.build_rhs(u0, f, tau)
    trr = oaao.true_relative_residual(K, tau, Fh, host(U))
    assert info["true_rel_res"] <= 1e-10 and trr <= 1e-10, (info, trr)
    Useq = oaao.sequential_bdf2(K, tau, u0, f)
    bound = 1e-10 if prec == aao.AAO_PREC_FP64 else 1e-9
    assert rel(host(U), Useq) <= bound, rel(host(U), Useq)


@pytest.mark.parametrize("prec,nt_max", [(aao.AAO_PREC_MIXED, 4096), (aao.AAO_PREC_FP64, 2048)])
def test_largest_accepted_nt_solves_and_the_next_is_rejected(prec, nt_max):
    # The time DFTs of Steps (a)/(c) keep all Nt rows of a column tile in shared memory (227 KB per block on
    # this GPU): the largest accepted Nt solves like any other, the next power of two is refused up front.
    M, alpha = 15, 1.6
    u0, f, U, info = solve_case(M, nt_max, alpha, prec, aao.AAO_INNER_TAU, recipe="sine1_uniform")
    K = jac(M, alpha)
    tau = 1.0 / nt_max
    Useq = oaao.sequential_bdf2(K, tau, u0, f)
    assert info["true_rel_res"] <= 1e-10, info
    assert rel(U, Useq) <= (1e-9 if prec == aao.AAO_PREC_MIXED else 1e-10), rel(U, Useq)
    with pytest.raises(aao.AaoError) as e:
        aao.Plan(M, 2 * nt_max, alpha, prec=prec)
    assert e.value.status == aao.AAO_EINVAL and "at most %d" % nt_max in str(e.value)


def breakdown_rhs(prec, Nt=8, M=2, alpha=1.5):
    """A crafted right-hand side whose frequency-1 shifted system has b^T A^{-1} b = 0 (complex b): at
    M = 2 the Strang circulant equals T, so COCG's first rho = r^T z = b^T A^{-1} b vanishes up to
    rounding.  Returns (F, eps)."""
    tau = 1.0 / Nt
    c = tau / (1.0 / (M + 1)) ** alpha
    eps = mixed_eps(tau) if prec == aao.AAO_PREC_MIXED else oprec.default_eps(tau)
    lam = oprec.eigenvalues_C_eps(Nt, eps)[1]
    g = fcd.fcd_weights(alpha, M)
    a, cp = lam + c * g[0], c * g[1]
    b = np.array([1.0, (cp + np.sqrt(cp * cp - a * a + 0j)) / a])  # a (b0^2 + b1^2) - 2 cp b0 b1 = 0
    k = np.arange(Nt)
    F = (eps ** (-k / Nt))[:, None] * (2.0 / Nt) * np.real(b[None, :] * np.exp(-2j * np.pi * k / Nt)[:, None])
    zh = oprec.time_dft_half(F, eps)  # Step (a) gives b at n = 1 and zero elsewhere
    np.testing.assert_allclose(zh[1], b, atol=1e-12)
    assert np.abs(np.delete(zh, 1, axis=0)).max() < 1e-12
    return F, eps


@pytest.mark.parametrize("prec", [aao.AAO_PREC_MIXED, aao.AAO_PREC_FP64])
def test_cocg_breakdown_is_detected_and_fgmres_still_converges(prec):
    # The relative breakdown test (|u^T w| <= 64 u ||u|| ||w||) must report the crafted breakdown
    # (status_detail = AAO_EBREAKDOWN), and flexible GMRES absorbs the failed inner solve.
    Nt, M, alpha = 8, 2, 1.5
    tau = 1.0 / Nt
    F, eps = breakdown_rhs(prec, Nt, M, alpha)
    with aao.Plan(M, Nt, alpha, prec=prec, inner=aao.AAO_INNER_STRANG, matvec=aao.AAO_MATVEC_FFT64) as plan:
        U = torch.zeros((Nt, M), dtype=torch.float64, device=DEV)
        info = plan.gmres_solve(cu(F), U)
    assert info["status_detail"] == aao.AAO_EBREAKDOWN, info
    K = jac(M, alpha)
    assert oaao.true_relative_residual(K, tau, F, host(U)) <= 1e-10, info
    np.testing.assert_allclose(host(U), np.linalg.solve(oaao.assemble_all_at_once(K, Nt, tau), F.ravel()).reshape(Nt, M),
                               rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("prec", [aao.AAO_PREC_MIXED, aao.AAO_PREC_FP64])
def test_inner_record_names_the_system_that_broke_down(prec):
    # Step (a) of the crafted right-hand side is nonzero at frequency 1 only (elsewhere it is zero or at
    # rounding level): the record of one preconditioner application shows a breakdown there and
    # convergence everywhere else (at most M = 2 iterations; none for an exactly zero right-hand side).
    Nt, M, alpha = 8, 2, 1.5
    F, _ = breakdown_rhs(prec, Nt, M, alpha)
    with aao.Plan(M, Nt, alpha, prec=prec, inner=aao.AAO_INNER_STRANG, matvec=aao.AAO_MATVEC_FFT64) as plan:
        z = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(F), z)
        it, fl = plan.inner_record()
    assert it.shape == (Nt // 2 + 1,) and fl[1] == 2, (it, fl)
    assert (np.delete(fl, 1) == 0).all() and (np.delete(it, 1) <= M).all(), (it, fl)


def test_tiny_right_hand_side_is_no_breakdown():
    # COCG is scale invariant: a right-hand side of 1e-17 N(0, 1) entries (squares near the FP32 underflow
    # threshold) converges like any other and gives z = 1e-17 P_eps^{-1} v' (the mixed path normalises
    # each shifted system's right-hand side by its 1-norm before the iteration).
    Nt, M, alpha = 8, 2, 1.5
    v = workloads.random_vector(Nt, M, seed=7)
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED, matvec=aao.AAO_MATVEC_FFT64) as plan:
        z1 = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z1)
        z2 = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(1e-17 * v), z2)
        it, fl = plan.inner_record()
    assert (fl == 0).all() and (it >= 1).all(), (it, fl)
    assert rel(1e17 * host(z2), host(z1)) <= 1e-5, rel(1e17 * host(z2), host(z1))


@pytest.mark.parametrize("inner", [aao.AAO_INNER_STRANG, aao.AAO_INNER_TAU, aao.AAO_INNER_TAU_DIRECT])
def test_inner_record_of_a_generic_apply(inner):
    M, Nt, alpha = 255, 32, 1.8
    v = workloads.random_vector(Nt, M, seed=6)
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED, inner=inner) as plan:
        z = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        it, fl = plan.inner_record()
        with pytest.raises(aao.AaoError):
            record_with_wrong_count(plan)
    assert (fl == 0).all(), fl
    if inner == aao.AAO_INNER_TAU_DIRECT:
        assert (it == 0).all(), it
    else:
        assert it.min() >= 1 and it.max() <= 200, it


def record_with_wrong_count(plan):
    import ctypes
    n = plan.Nt // 2
    buf = np.zeros(n + 1, dtype=np.int32)
    aao._check(aao.load().aao_plan_get_inner_record(plan.handle, n, buf.ctypes.data_as(ctypes.c_void_p), None),
               plan.handle)
