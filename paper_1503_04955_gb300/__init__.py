"""GB300 (sm_103a) DKSS integer multiplication: Python binding of libdkss.so.

The arithmetic runs in hand-written CUDA kernels behind the C ABI declared in
include/dkss.h; this package builds the library (buildlib.py) and marshals
arguments to it (binding.py).
"""
from .binding import Plan, Batch, DkssError, plan_rho, plan_choose, proth_ring, plan_proth_rho, plan_candidates, load, lib_path, mul_batch, ll_step, EXPORTS  # noqa: F401
from .binding import TUNE_RULE, DEBUG_CHECKS, FORM_INT8TC, FAULT_RANGE, ARITH_MONT, RMUL_DIRECT  # noqa: F401
from .buildlib import build  # noqa: F401
