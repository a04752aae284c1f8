"""GB300 (sm_103a) implementation of Tygert's randomized minimal-norm solver
(arXiv:0905.4745) behind the C ABI of include/minnorm.h.

    from paper_0905_4745_gb300 import minnorm as mn
    plan = mn.minnorm_plan_create(m, n, dtype=mn.C128, precision=mn.MIXED, seed=1)
    mn.minnorm_sketch(plan, A)                  # Steps 1-2: Y = T A^*, Y P = Q R
    st, info = mn.minnorm_solve(plan, A, b, 1e-12, x)   # Steps 3-5
    mn.minnorm_plan_destroy(plan)
"""
from . import minnorm  # noqa: F401
