"""Plain FP64 CPU oracle for the stabilised fermion log-weight of the Holstein model
and for the symmetric effective-model Markov chain of self-learning Monte Carlo.

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously-correct reference that
the CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The product
path (the C-ABI library and its Python binding) never imports, links or calls it, and
this package imports nothing from the product package.

Every function cites the passage of the paper (arXiv:1802.06177, "Symmetry enforced
self-learning Monte Carlo method applied to the Holstein model") it follows. Where the
paper is silent (the UDT stabilisation, the proposal distribution, the random-number
layout) the docstring states the reading taken.

Parity pins (tests/test_oracle_*.py, run with ``-m "not gpu"``): closed forms at
lambda=0, uniform and static staggered fields and t=0, brute-force LU of the NL x NL
fermion matrix, particle-hole / translation / time-reversal invariances, the Z2 mirror
of E_eff, exact Boltzmann sampling on tiny systems, exact regression recovery, the
J_k = 1/(2 dtau^2) entry of Table S1, and exact detailed balance of the modified Wolff
cluster move (enumeration of all bond-activation patterns on small lattices). Parity is unpinned only for the physics values of
S(pi,pi) at the benchmark parameters (the paper prints none there).
"""
from .params import HolsteinParams  # noqa: F401
