"""CPU FP64 oracle for the all-at-once BDF2 system of the Riesz fractional
diffusion equation (Gu, Zhao, Zhao, Carpentieri, Huang, arXiv:2003.07020).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg (``cpu_baseline`` / ``--impl reference``) call it.  It shares
no code with the CUDA path (``paper_2003_07020_gb300``); the only module both
sides use is the seeded input generator ``paper_2003_07020_gb300.workloads``,
which holds none of the method's arithmetic.

Everything is plain numpy / scipy in float64 (complex128), written to be
checked against the paper by eye:

* :mod:`oracle.fcd`      -- weights g_k (Eq. 2.4), the Toeplitz Jacobian (Sec. 2.1)
* :mod:`oracle.aao`      -- the all-at-once system (Eqs. 11-12), its matvec
                            (Sec. 3.2) and sequential BDF2 time stepping (Eq. 1.2)
* :mod:`oracle.precond`  -- the eps-circulant preconditioner (Eq. 1.11, Sec. 3.1)
                            applied exactly by the three steps (a)-(c), the
                            Strang circulant and preconditioned COCG for Step-(b)
* :mod:`oracle.gmres`    -- restarted right-preconditioned (F)GMRES (Sec. 4)
* :mod:`oracle.examples` -- the manufactured solutions of Examples 1 and 2 (Sec. 4)

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py`` except where the
docstring says "parity unpinned".
"""
