"""FP64 CPU oracle for the localized-collision Projective Dynamics iteration.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the test-suite, the smoke check in the repository's
entry module and the CPU-baseline leg of the benchmark use it.  It shares no
code with the CUDA library; the two meet only in the seeded scene generators.
"""
from .pd_oracle import *  # noqa: F401,F403
