"""Batched solves (many independent 1D instances of different M, Nt, alpha,
kappa in one aao_solve_batched call) against single solves and the oracle."""
import numpy as np
import pytest

from paper_2003_07020_gb300 import aao, workloads
from oracle import aao as oaao, fcd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def setup(inst, prec=aao.AAO_PREC_MIXED):
    M, Nt = inst["M"], inst["Nt"]
    plan = aao.Plan(M, Nt, inst["alpha"], kappa=inst["kappa"], prec=prec)
    u0, f = workloads.make_inputs(M, Nt, seed=inst["seed"])
    F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
    plan.build_rhs(torch.from_numpy(u0).to(DEV), torch.from_numpy(f).to(DEV), F)
    return plan, F, u0, f


def test_batched_equals_single_solves_and_oracle():
    insts = workloads.batched_instances(8, seed=3, Ms=(63, 127, 255), Nts=(16, 32, 64))
    plans, Fs, Us, data = [], [], [], []
    for inst in insts:
        p, F, u0, f = setup(inst)
        plans.append(p)
        Fs.append(F)
        Us.append(torch.zeros_like(F))
        data.append((u0, f))
    infos = aao.solve_batched(plans, Fs, Us, max_workers=4)
    torch.cuda.synchronize()
    for inst, p, F, U, info, (u0, f) in zip(insts, plans, Fs, Us, infos, data):
        Us1 = torch.zeros_like(F)
        info1 = p.gmres_solve(F, Us1)
        # the same deterministic kernels on another stream: identical results
        assert torch.equal(U, Us1), inst
        assert info["outer_iters"] == info1["outer_iters"]
        M, Nt = inst["M"], inst["Nt"]
        K = fcd.jacobian_1d(inst["alpha"], inst["kappa"], M, 1.0 / (M + 1))
        Useq = oaao.sequential_bdf2(K, 1.0 / Nt, u0, f)
        Uh = U.cpu().numpy()
        assert info["true_rel_res"] <= 1e-10
        assert np.linalg.norm(Uh - Useq) <= 1e-9 * np.linalg.norm(Useq), inst
    for p in plans:
        p.close()


def test_batched_reports_failures_without_stopping_others():
    insts = workloads.batched_instances(3, seed=4, Ms=(63,), Nts=(16,))
    plans, Fs, Us = [], [], []
    for inst in insts:
        p, F, _, _ = setup(inst)
        plans.append(p)
        Fs.append(F)
        Us.append(torch.zeros_like(F))
    Fs[1][0, 0] = float("nan")
    infos = aao.solve_batched(plans, Fs, Us, raise_on_error=False)
    assert infos[0]["true_rel_res"] <= 1e-10 and infos[2]["true_rel_res"] <= 1e-10
    for p in plans:
        p.close()


def test_lockstep_batched_is_one_step_b_launch_per_step_and_equals_single_solves():
    # All instances share the CTA size of the Step (b) kernel (the lockstep launch uses the largest of the
    # plans'), so every kernel computes exactly what the single solves compute: bit-equal results.
    insts = workloads.batched_instances(6, seed=5, Ms=(63, 127, 255, 511), Nts=(16, 32, 64))
    plans, Fs, Us, data = [], [], [], []
    for inst in insts:
        M, Nt = inst["M"], inst["Nt"]
        p = aao.Plan(M, Nt, inst["alpha"], kappa=inst["kappa"], prec=aao.AAO_PREC_MIXED, cocg_threads=128)
        u0, f = workloads.make_inputs(M, Nt, seed=inst["seed"])
        F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
        p.build_rhs(torch.from_numpy(u0).to(DEV), torch.from_numpy(f).to(DEV), F)
        plans.append(p)
        Fs.append(F)
        Us.append(torch.zeros_like(F))
        data.append((u0, f))
    for p in plans:
        p.get_profile(reset=True)
    infos = aao.solve_batched(plans, Fs, Us, max_workers=0)
    torch.cuda.synchronize()
    step_b = sum(p.get_profile(reset=True)["cocg"][1] for p in plans)
    # one restart cycle each (they converge within 20 steps): the lockstep runs max(outer_iters) steps,
    # each with a single Step (b) launch for every instance still iterating
    assert max(i["cycles"] for i in infos) == 1
    assert step_b == max(i["outer_iters"] for i in infos), (step_b, [i["outer_iters"] for i in infos])
    for inst, p, F, U, info, (u0, f) in zip(insts, plans, Fs, Us, infos, data):
        U1 = torch.zeros_like(F)
        info1 = p.gmres_solve(F, U1)
        assert torch.equal(U, U1), inst
        assert info["outer_iters"] == info1["outer_iters"] and info["inner_iters_sum"] == info1["inner_iters_sum"]
        M, Nt = inst["M"], inst["Nt"]
        K = fcd.jacobian_1d(inst["alpha"], inst["kappa"], M, 1.0 / (M + 1))
        Useq = oaao.sequential_bdf2(K, 1.0 / Nt, u0, f)
        assert info["true_rel_res"] <= 1e-10
        assert np.linalg.norm(U.cpu().numpy() - Useq) <= 1e-9 * np.linalg.norm(Useq), inst
    for p in plans:
        p.close()


def test_lockstep_batched_reports_failures_without_stopping_others():
    insts = workloads.batched_instances(3, seed=4, Ms=(63,), Nts=(16,))
    plans, Fs, Us = [], [], []
    for inst in insts:
        p, F, _, _ = setup(inst)
        plans.append(p)
        Fs.append(F)
        Us.append(torch.zeros_like(F))
    Fs[1][0, 0] = float("nan")
    infos = aao.solve_batched(plans, Fs, Us, max_workers=0, raise_on_error=False)
    assert infos[0]["true_rel_res"] <= 1e-10 and infos[2]["true_rel_res"] <= 1e-10
    for p in plans:
        p.close()
