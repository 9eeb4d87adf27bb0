"""FP64 CPU oracle of the ABCS hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline/reference
legs may import this package.  The CUDA library never does, and this package
never imports the library.
"""
from .abcs_oracle import *  # noqa: F401,F403
from .abcs_oracle import ZZ, BBV, DD, VARIANTS  # noqa: F401
