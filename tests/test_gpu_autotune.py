"""Launch-shape autotuning of the Step (b) kernel: every admissible CTA size of the
register-resident FP32 COCG kernel gives the same solve (to FP32 reduction order),
and the autotuned choice is admissible and cached per problem shape."""
import numpy as np
import pytest

from paper_2003_07020_gb300 import aao, workloads
from oracle import aao as oaao, fcd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("inner", [aao.AAO_INNER_STRANG, aao.AAO_INNER_TAU])
def test_every_cta_size_solves_the_same_problem(inner):
    M, Nt, alpha = 255, 32, 1.6
    u0, f = workloads.make_inputs(M, Nt, seed=4)
    K = fcd.jacobian_1d(alpha, 1.0, M, 1.0 / (M + 1))
    Useq = oaao.sequential_bdf2(K, 1.0 / Nt, u0, f)
    its = []
    for nt in (64, 128, 256, 512):
        with aao.Plan(M, Nt, alpha, inner=inner, cocg_threads=nt) as plan:
            assert plan.cocg_threads == nt
            F = torch.empty((Nt, M), dtype=torch.float64, device=DEV)
            plan.build_rhs(cu(u0), cu(f), F)
            U = torch.zeros_like(F)
            info = plan.gmres_solve(F, U)
        assert info["true_rel_res"] <= 1e-10
        Uh = U.cpu().numpy()
        assert np.linalg.norm(Uh - Useq) <= 1e-9 * np.linalg.norm(Useq), nt
        its.append(info["outer_iters"])
    assert max(its) - min(its) <= 1, its


def test_autotuned_choice_is_admissible_and_cached():
    for M, lo in ((63, 64), (1023, 64), (2047, 128), (4095, 256)):
        a = aao.Plan(M, 16, 1.5)
        b = aao.Plan(M, 16, 1.7)  # same shape: the cached choice
        assert lo <= a.cocg_threads <= 512 and a.cocg_threads & (a.cocg_threads - 1) == 0, (M, a.cocg_threads)
        assert b.cocg_threads == a.cocg_threads
        a.close()
        b.close()
    # above M = 4096 the Strang systems go to the tensor-memory kernel unless a CTA size is given
    with aao.Plan(8191, 16, 1.5) as a, aao.Plan(8191, 16, 1.5, cocg_threads=512) as b:
        assert a.cocg_threads == aao.AAO_COCG_TMEM and b.cocg_threads == 512
    with aao.Plan(8191, 16, 1.5, inner=aao.AAO_INNER_TAU) as c:
        assert c.cocg_threads == 512
    with aao.Plan(8191, 16, 1.5, prec=aao.AAO_PREC_FP64) as p64:
        assert p64.cocg_threads == 0
