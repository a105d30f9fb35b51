"""GB300-native hot path of symmetry-enforced self-learning Monte Carlo for the 2D
Holstein model (arXiv:1802.06177): stabilised ln det(I + B_L ... B_1), the equal-time
Green's function, the symmetric effective model and its cumulative-update Markov chain.

The compute lives in libslmc.so (hand-written CUDA for sm_103a behind the C ABI of
include/slmc.h); ``paper_1802_06177_gb300.slmc`` is a thin ctypes binding over it.
Importing the package does not load the library; constructing a ``Context`` does, and
fails loudly if the library is missing.
"""
__all__ = ["slmc", "inputs", "workloads"]
