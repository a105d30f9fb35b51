"""CDW structure factor from the equal-time Green's function (oracle; test
infrastructure only).

Sec. "Results": S_CDW = (1/N) sum_ij (-1)^(i+j) (<n_i n_j> - <n_i><n_j>).
Per configuration, with G_ij = <c_i c_j^dagger> identical for both spins, Wick's theorem
gives <n_i n_j> = 4 (1 - G_ii)(1 - G_jj) + 2 (delta_ij - G_ji) G_ij. Reading taken:
<n_i><n_j> uses Monte Carlo averages, whose staggered sum vanishes at half filling, so
the per-configuration estimator keeps only the first part.
"""
import numpy as np

from .lattice import staggered_sign


def s_cdw(p, G):
    s = staggered_sign(p.Lx, p.Ly)
    G = np.asarray(G, dtype=np.float64)
    N = p.N
    n = 1.0 - np.diag(G)
    nn = 4.0 * np.outer(n, n) + 2.0 * (np.eye(N) - G.T) * G
    return float(s @ nn @ s) / N
