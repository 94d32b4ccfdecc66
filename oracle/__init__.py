"""CPU oracle of the multilevel Chebyshev-Hutchinson trace estimator.

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is
checked against.  Only the test suite, the package smoke check and the
benchmark's CPU-baseline / reference arm may import it; the product path never
does.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
