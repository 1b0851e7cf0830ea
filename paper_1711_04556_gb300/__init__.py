"""GB300 (sm_103a) tabu search for the Resource Constrained Project Scheduling
Problem, after Bukata, Sucha and Hanzalek (J. Parallel Distrib. Comput. 77,
2015).

``rcpsp.Solver`` is the Python face of the C library in include/rcpsp.h;
``instances`` draws seeded synthetic workloads.  Importing the package does
not need the CUDA library; the first Solver does and fails loudly without
it.
"""
from .instances import Instance, config_batch, generate, level_keys, table1_instance  # noqa: F401
from .rcpsp import EVAL_AUTO, EVAL_CAPACITY, EVAL_TIME, RcpspError, Solver  # noqa: F401
