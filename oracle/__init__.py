"""FP64 CPU oracle of the contact-smoothed quasi-static simulator (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg / reference arm may import
this package.  The CUDA path neither imports it nor shares any code with it.
"""
from . import sim, grad  # noqa: F401
