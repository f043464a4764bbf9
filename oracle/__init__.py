"""Plain FP64 CPU oracle of the VP-LBM time step (arXiv 1812.05401).

TEST INFRASTRUCTURE ONLY. The CUDA library is checked against this package; it
shares no code with it. Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import it.
"""
from .oracle import *  # noqa: F401,F403
