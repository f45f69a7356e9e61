"""GB300 (sm_103a) solver for the all-at-once BDF2 system of the Riesz
fractional diffusion equation (arXiv:2003.07020).

* :mod:`paper_2003_07020_gb300.aao`       -- ctypes binding of ``include/aao.h``
* :mod:`paper_2003_07020_gb300.workloads` -- seeded synthetic inputs
* :mod:`paper_2003_07020_gb300.build`     -- nvcc build of ``libaao.so``
"""
from . import workloads  # noqa: F401
