"""GPU parity of the 2D path (K = I (x) K_x + K_y (x) I, x fastest; Eq. 4.2 on
(0,1)^2) against the CPU oracle, through the C ABI.

Tolerances as in test_gpu_parity.py: matvec 1e-13 relative (FP64 FFT
rounding); preconditioner FP64 residual 1e-10 / z 1e-9 and mixed
4 (t + 64 u32) / eps; solve true residual <= 1e-10 and forward error 1e-10
(FP64) or 1e-9 (mixed) against sequential BDF2 by fast diagonalisation.
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


def mixed_eps(tau):
    """The library's default circulant parameter for the mixed path: max(min(0.5, 0.5 tau), 1/16)."""
    return max(min(0.5, 0.5 * tau), 1.0 / 16)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def jacs(Mx, My, ax, ay, kx=1.0, ky=1.0):
    return (fcd.jacobian_1d(ax, kx, Mx, 1.0 / (Mx + 1)), fcd.jacobian_1d(ay, ky, My, 1.0 / (My + 1)))


CASES = [(15, 7, 8, 1.3, 1.7), (31, 63, 16, 1.5, 1.2), (7, 3, 4, 1.9, 1.1), (255, 255, 4, 1.3, 1.7)]


@pytest.mark.parametrize("kind", [aao.AAO_MATVEC_NTT, aao.AAO_MATVEC_FFT64])
@pytest.mark.parametrize("Mx,My,Nt,ax,ay", CASES)
def test_matvec_2d(Mx, My, Nt, ax, ay, kind):
    # exact-integer line convolutions (default) and FP64 FFTs: 1e-13 in norm, and for the exact form every
    # element within 1e-13 of the largest (the 58-bit level quantisation is the only rounding before FP64)
    v = np.random.default_rng(Mx + My).standard_normal((Nt, My, Mx))
    with aao.Plan(Mx, Nt, ax, My=My, alpha_y=ay, matvec=kind) as plan:
        w = torch.empty((Nt, My, Mx), dtype=torch.float64, device=DEV)
        plan.matvec(cu(v), w)
        torch.cuda.synchronize()
    Kx, Ky = jacs(Mx, My, ax, ay)
    want = oaao.matvec_2d(Kx, Ky, 1.0 / Nt, v)
    assert rel(host(w), want) <= 1e-13
    if kind == aao.AAO_MATVEC_NTT:
        assert np.abs(host(w) - want).max() <= 1e-13 * np.abs(want).max()


def test_gmres_2d_with_the_fp64_fft_matvec():
    Mx, My, Nt, ax, ay = 31, 15, 16, 1.4, 1.6
    u0, f = workloads.make_inputs_2d(Mx, My, Nt, seed=3)
    Kx, Ky = jacs(Mx, My, ax, ay)
    Useq = oaao.sequential_bdf2_2d(Kx, Ky, 1.0 / Nt, u0, f)
    with aao.Plan(Mx, Nt, ax, My=My, alpha_y=ay, matvec=aao.AAO_MATVEC_FFT64) as plan:
        F = torch.empty((Nt, My, Mx), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        U = torch.zeros_like(F)
        info = plan.gmres_solve(F, U)
    assert info["true_rel_res"] <= 1e-10, info
    assert rel(host(U), Useq) <= 1e-9


INNERS = [aao.AAO_INNER_STRANG, aao.AAO_INNER_TAU]


@pytest.mark.parametrize("Mx,My,Nt,ax,ay", CASES[:3])
@pytest.mark.parametrize("inner", INNERS)
def test_precond_2d_fp64(Mx, My, Nt, ax, ay, inner):
    v = np.random.default_rng(3).standard_normal((Nt, My, Mx))
    tau = 1.0 / Nt
    eps = oprec.default_eps(tau)
    with aao.Plan(Mx, Nt, ax, My=My, alpha_y=ay, prec=aao.AAO_PREC_FP64, inner=inner) as plan:
        z = torch.empty((Nt, My, Mx), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        torch.cuda.synchronize()
    Kx, Ky = jacs(Mx, My, ax, ay)
    Z = host(z)
    assert rel(oprec.P_eps_matvec_2d(Kx, Ky, tau, eps, Z), v) <= 1e-10
    assert rel(Z, oprec.precond_apply_2d(Kx, Ky, tau, eps, v)) <= 1e-9


@pytest.mark.parametrize("Mx,My,Nt,ax,ay", CASES[:3])
@pytest.mark.parametrize("inner", INNERS)
def test_precond_2d_mixed(Mx, My, Nt, ax, ay, inner):
    v = np.random.default_rng(4).standard_normal((Nt, My, Mx))
    tau = 1.0 / Nt
    eps = mixed_eps(tau)
    with aao.Plan(Mx, Nt, ax, My=My, alpha_y=ay, prec=aao.AAO_PREC_MIXED, inner=inner) as plan:
        z = torch.empty((Nt, My, Mx), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        torch.cuda.synchronize()
    Kx, Ky = jacs(Mx, My, ax, ay)
    err = rel(host(z), oprec.precond_apply_2d(Kx, Ky, tau, eps, v))
    assert err <= 4 * (1e-6 + 64 * 2.0 ** -24) / eps, err


@pytest.mark.parametrize("prec,bound", [(aao.AAO_PREC_FP64, 1e-10), (aao.AAO_PREC_MIXED, 1e-9)])
@pytest.mark.parametrize("Mx,My,Nt,ax,ay", [(31, 15, 16, 1.3, 1.7), (63, 63, 32, 1.5, 1.2)])
@pytest.mark.parametrize("inner", INNERS)
@pytest.mark.parametrize("graphs", [1, 0])
def test_gmres_2d_matches_time_stepping(Mx, My, Nt, ax, ay, prec, bound, inner, graphs):
    u0, f = workloads.make_inputs_2d(Mx, My, Nt, seed=5)
    tau = 1.0 / Nt
    with aao.Plan(Mx, Nt, ax, My=My, alpha_y=ay, prec=prec, inner=inner, use_graphs=graphs) as plan:
        F = torch.empty((Nt, My, Mx), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        U = torch.zeros_like(F)
        info = plan.gmres_solve(F, U)
    Kx, Ky = jacs(Mx, My, ax, ay)
    Useq = oaao.sequential_bdf2_2d(Kx, Ky, tau, u0, f)
    Fh = oaao.build_rhs(u0, f, tau)
    R = Fh - oaao.matvec_2d(Kx, Ky, tau, host(U))
    trr = np.linalg.norm(R) / np.linalg.norm(Fh)
    assert info["true_rel_res"] <= 1e-10 and trr <= 1e-10, (info, trr)
    assert rel(host(U), Useq) <= bound, (rel(host(U), Useq), info)


def test_gmres_2d_full_size_config():
    # 255 x 255 interior points, Nt = 256, alphas (1.3, 1.7), kappa = 1
    Mx = My = 255
    Nt = 256
    ax, ay = 1.3, 1.7
    u0, f = workloads.make_inputs_2d(Mx, My, Nt, seed=0)
    tau = 1.0 / Nt
    with aao.Plan(Mx, Nt, ax, My=My, alpha_y=ay, prec=aao.AAO_PREC_MIXED) as plan:
        F = torch.empty((Nt, My, Mx), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        U = torch.zeros_like(F)
        info = plan.gmres_solve(F, U)
    Kx, Ky = jacs(Mx, My, ax, ay)
    Fh = oaao.build_rhs(u0, f, tau)
    trr = np.linalg.norm(Fh - oaao.matvec_2d(Kx, Ky, tau, host(U))) / np.linalg.norm(Fh)
    assert info["true_rel_res"] <= 1e-10 and trr <= 1e-10, (info, trr)
    Useq = oaao.sequential_bdf2_2d(Kx, Ky, tau, u0, f)
    assert rel(host(U), Useq) <= 1e-9, (rel(host(U), Useq), info)


@pytest.mark.parametrize("Mx,My,Nt", [(15, 7, 8), (31, 63, 4)])
def test_strang2d_preconditioner_after_one_cocg_step(Mx, My, Nt):
    # With one COCG iteration per system the GPU's Step (b) returns x_n = a_n P_n^{-1} b_n with
    # P_n = lambda_n I + I (x) c_x S_x + c_y S_y (x) I (the 2D Strang BCCB circulant) and
    # a_n = (b_n^T z_n) / (z_n^T A_n z_n), z_n = P_n^{-1} b_n: this pins the BCCB inverse itself against the
    # oracle's (FP64 throughout, so to rounding).
    ax, ay = 1.4, 1.8
    tau = 1.0 / Nt
    eps = oprec.default_eps(tau)
    v = np.random.default_rng(Mx + My).standard_normal((Nt, My, Mx))
    with aao.Plan(Mx, Nt, ax, My=My, alpha_y=ay, prec=aao.AAO_PREC_FP64, inner=aao.AAO_INNER_STRANG,
                  inner_maxit=1) as plan:
        z = torch.empty((Nt, My, Mx), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        torch.cuda.synchronize()
    Kx, Ky = jacs(Mx, My, ax, ay)
    hx, hy = 1.0 / (Mx + 1), 1.0 / (My + 1)
    gx = (tau / hx ** ax) * fcd.fcd_weights(ax, Mx)
    gy = (tau / hy ** ay) * fcd.fcd_weights(ay, My)
    zh = oprec.time_dft_half(v, eps).reshape(Nt // 2 + 1, My, Mx)
    lam = oprec.eigenvalues_C_eps(Nt, eps)
    K = np.kron(np.eye(My), Kx) + np.kron(Ky, np.eye(Mx))
    xh = np.empty_like(zh)
    for n in range(Nt // 2 + 1):
        b = zh[n]
        zz = oprec.strang2d_inverse(gx, gy, Mx, My, lam[n])(b)
        Az = (lam[n] * np.eye(Mx * My) - tau * K) @ zz.ravel()
        xh[n] = (b.ravel() @ zz.ravel()) / (zz.ravel() @ Az) * zz
    want = oprec.time_idft_half(xh, eps, Nt)
    assert rel(host(z), want) <= 1e-11, rel(host(z), want)
