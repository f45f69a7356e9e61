"""The no-allocation preconditioner entry point against the plan-based one.

aao_bc_precond_apply_noalloc is for callers that cannot call cudaMalloc
(for example code that runs inside another library's memory pool or that
must not synchronise the device through an allocation): it needs no plan and
keeps its scratch in a fixed device array of the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_07020_gb300 import aao, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,Nt,alpha,inner", [(63, 64, 1.5, aao.AAO_INNER_STRANG),
                                              (1023, 32, 1.8, aao.AAO_INNER_TAU),
                                              (8191, 256, 1.5, aao.AAO_INNER_STRANG)])  # about 9 of the 16 MiB
def test_noalloc_matches_plan_apply_twice(M, Nt, alpha, inner):
    lib = aao.load()
    v = torch.from_numpy(workloads.random_vector(Nt, M, seed=11)).to("cuda:0")
    prob = aao.AaoProblem(1, M, Nt, 1.0, alpha, 1.0, 0.0)
    opts = aao.default_opts(aao.AAO_PREC_MIXED, inner=inner)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with aao.Plan(M, Nt, alpha, opts=opts) as plan:
        ref = torch.empty_like(v)
        plan.bc_precond_apply(v, ref)
    for _ in range(2):  # two calls in a row share the same scratch array
        z = torch.full_like(v, float("nan"))
        st = lib.aao_bc_precond_apply_noalloc(ctypes.byref(prob), ctypes.byref(opts), ctypes.c_void_p(v.data_ptr()),
                                              ctypes.c_void_p(z.data_ptr()), stream)
        assert st == aao.AAO_OK, lib.aao_last_error(None)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(z - ref) / torch.linalg.norm(ref)).item()
        # same kernels and tables as the plan path; the mixed-path tolerance of the parity tests
        eps = max(min(0.5, 0.5 / Nt), 1.0 / 16)
        assert err <= 4 * (1e-6 + 64 * 2.0 ** -24) / eps, err


def test_noalloc_rejects_oversized_problem():
    lib = aao.load()
    prob = aao.AaoProblem(1, 8191, 1024, 1.0, 1.5, 1.0, 0.0)   # 513 * 8191 * 8 B > 16 MiB
    opts = aao.default_opts(aao.AAO_PREC_MIXED)
    v = torch.zeros((1024, 8191), dtype=torch.float64, device="cuda:0")
    st = lib.aao_bc_precond_apply_noalloc(ctypes.byref(prob), ctypes.byref(opts), ctypes.c_void_p(v.data_ptr()),
                                          ctypes.c_void_p(v.data_ptr()), None)
    assert st == aao.AAO_EINVAL
    assert b"16 MiB" in lib.aao_last_error(None)
