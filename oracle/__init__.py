"""FP64 CPU oracle for the SEM elliptic path (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package; the library itself never does.
"""
from .sem_oracle import *  # noqa: F401,F403
