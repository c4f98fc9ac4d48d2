"""CPU oracle for comparator-based K-NN descent with the KL comparator.

Test infrastructure only: the test suite, the smoke check and the benchmark's
CPU-baseline leg are its only users.  The product path never imports it.
"""
from .oracle import *  # noqa: F401,F403
