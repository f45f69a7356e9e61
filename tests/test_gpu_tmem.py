"""Step (b) by the tensor-memory kernel (cocg_tm.cu: COCG vectors in TMEM, 4096 < M <= 8191, Strang
preconditioner, the default there) against the oracle and against the register-resident kernel
(cocg_threads = 512) on the same inputs."""
import numpy as np
import pytest

from paper_2003_07020_gb300 import aao, workloads
from oracle import aao as oaao, fcd, precond as oprec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def mixed_eps(tau):
    return max(min(0.5, 0.5 * tau), 1.0 / 16)


def apply(M, Nt, alpha, v, ct):
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED, cocg_threads=ct) as plan:
        assert plan.cocg_threads == ct
        z = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.bc_precond_apply(cu(v), z)
        it, fl = plan.inner_record()
    return z.cpu().numpy(), it, fl


@pytest.mark.parametrize("M,Nt,alpha", [(4097, 16, 1.5), (8191, 8, 1.8)])
def test_tmem_kernel_agrees_with_register_kernel(M, Nt, alpha):
    # Same operator, same recurrence: the two kernels differ only in FP32 rounding (transform order), so
    # the preconditioned vectors agree to the inner tolerance amplified by cond(V_eps) = 1/eps and the
    # iteration counts by at most two per system.
    v = workloads.random_vector(Nt, M, seed=11)
    zt, itt, flt = apply(M, Nt, alpha, v, aao.AAO_COCG_TMEM)
    zr, itr, flr = apply(M, Nt, alpha, v, 512)
    assert (flt == 0).all() and (flr == 0).all(), (flt, flr)
    assert np.abs(itt - itr).max() <= 2, (itt, itr)
    eps = mixed_eps(1.0 / Nt)
    assert rel(zt, zr) <= 4 * 1e-6 / eps, rel(zt, zr)


def test_tmem_residual_of_every_shifted_system():
    # As test_gpu_parity.py::test_precond_mixed_residual_of_every_shifted_system: the residual of each
    # shifted system recovered through exact FP64 Steps (a)/(c) is at most t + 16 u32 ||A_n|| ||x_n|| / ||y_n||.
    M, Nt, alpha = 4500, 16, 1.5
    v = workloads.random_vector(Nt, M, seed=12)
    z, its, fl = apply(M, Nt, alpha, v, aao.AAO_COCG_TMEM)
    assert (fl == 0).all(), fl
    tau = 1.0 / Nt
    eps = mixed_eps(tau)
    K = fcd.jacobian_1d(alpha, 1.0, M, 1.0 / (M + 1))
    mu = np.linalg.eigvalsh(K)
    lam = oprec.eigenvalues_C_eps(Nt, eps)
    Y = oprec.time_dft_half(v, eps)
    X = oprec.time_dft_half(z, eps)
    worst = 0.0
    for n in range(Nt // 2 + 1):
        ny = np.linalg.norm(Y[n])
        res = np.linalg.norm(Y[n] - (lam[n] * X[n] - tau * (K @ X[n]))) / ny
        bound = 1e-6 + 16 * 2.0 ** -24 * np.abs(lam[n] - tau * mu).max() * np.linalg.norm(X[n]) / ny
        worst = max(worst, res / bound)
        assert res <= bound, (n, res, bound, its[n])
    assert worst > 0.01, worst


def test_tmem_solve_matches_time_stepping():
    M, Nt, alpha = 4500, 16, 1.3
    u0, f = workloads.make_inputs(M, Nt, seed=13)
    K = fcd.jacobian_1d(alpha, 1.0, M, 1.0 / (M + 1))
    Useq = oaao.sequential_bdf2(K, 1.0 / Nt, u0, f)
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED) as plan:
        assert plan.cocg_threads == aao.AAO_COCG_TMEM
        F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        U = torch.zeros_like(F)
        info = plan.gmres_solve(F, U)
    assert info["true_rel_res"] <= 1e-10, info
    assert rel(U.cpu().numpy(), Useq) <= 1e-9, rel(U.cpu().numpy(), Useq)


def test_tmem_zero_tiny_and_nonfinite_right_hand_sides():
    M, Nt, alpha = 5000, 8, 1.6
    v = workloads.random_vector(Nt, M, seed=14)
    z0, it0, fl0 = apply(M, Nt, alpha, np.zeros((Nt, M)), aao.AAO_COCG_TMEM)
    assert not z0.any() and (it0 == 0).all() and (fl0 == 0).all()
    z1, _, _ = apply(M, Nt, alpha, v, aao.AAO_COCG_TMEM)
    z2, it2, fl2 = apply(M, Nt, alpha, 1e-17 * v, aao.AAO_COCG_TMEM)  # scale invariant (1-norm normalisation)
    assert (fl2 == 0).all() and (it2 >= 1).all()
    assert rel(1e17 * z2, z1) <= 1e-5, rel(1e17 * z2, z1)
    w = v.copy()
    w[3, 17] = np.nan
    _, _, fl3 = apply(M, Nt, alpha, w, aao.AAO_COCG_TMEM)
    assert (fl3 & 3 == 3).all(), fl3  # every frequency sees the NaN through Step (a)


def test_learned_warm_start_on_a_tensor_memory_plan():
    # The tensor-memory kernel takes no initial guess: with a model attached the plan's Step (b) runs on the
    # 512-thread register kernel, and the acceptance rule and FGMRES keep the result exact (random model).
    M, Nt, alpha = 4500, 16, 1.4
    u0, f = workloads.make_inputs(M, Nt, seed=15)
    K = fcd.jacobian_1d(alpha, 1.0, M, 1.0 / (M + 1))
    Useq = oaao.sequential_bdf2(K, 1.0 / Nt, u0, f)
    with aao.Plan(M, Nt, alpha, prec=aao.AAO_PREC_MIXED) as plan, aao.Fno(M, max_batch=Nt // 2 + 1, seed=2) as net:
        assert plan.cocg_threads == aao.AAO_COCG_TMEM
        F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        plan.build_rhs(cu(u0), cu(f), F)
        plan.set_warm_start(net)
        U = torch.zeros_like(F)
        info = plan.gmres_solve(F, U)
        plan.set_warm_start(None)
        U2 = torch.zeros_like(F)
        info2 = plan.gmres_solve(F, U2)  # back on the tensor-memory kernel
    for inf, u in ((info, U), (info2, U2)):
        assert inf["true_rel_res"] <= 1e-10, inf
        assert rel(u.cpu().numpy(), Useq) <= 1e-9
