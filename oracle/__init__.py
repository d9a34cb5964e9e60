"""CPU oracle for adaptive s-step CG (test infrastructure only).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline arm of
`bench.py` use this package. The solver library never imports it.
"""
from .ascg_oracle import *  # noqa: F401,F403
from .ascg_oracle import EPS, Operator, BasisParams  # noqa: F401
