"""Pins of the Green's function convention, the determinant and the CDW structure
factor against exact many-body traces in Fock space (2x2 lattice) and against the
free-fermion closed form."""
import itertools

import numpy as np
import scipy.linalg

from oracle import HolsteinParams
from oracle.fermion import fermion_logdet
from oracle.lattice import dispersion, exp_hopping, hopping_matrix, staggered_sign
from oracle.observables import s_cdw


def fock_operators(N):
    """Jordan-Wigner annihilation operators c_i on the 2^N Fock space of one spin."""
    I2, Z = np.eye(2), np.diag([1.0, -1.0])
    lower = np.array([[0.0, 1.0], [0.0, 0.0]])  # |0><1| annihilates
    ops = []
    for i in range(N):
        m = np.eye(1)
        for j in range(N):
            m = np.kron(m, Z if j < i else (lower if j == i else I2))
        ops.append(m)
    return ops


def test_fock_space_trace_green_function_and_cdw():
    p = HolsteinParams(2, 2, 6, lam=1.0, n_s=2, dtau=0.2)
    N = 4
    x = np.random.default_rng(8).normal(size=(N, p.L))
    c = fock_operators(N)
    n_op = [ci.T @ ci for ci in c]
    K = hopping_matrix(2, 2, p.t, p.mu)
    HK = sum(K[i, j] * c[i].T @ c[j] for i in range(N) for j in range(N))
    eK = scipy.linalg.expm(-p.dtau * HK)
    P = np.eye(2 ** N)
    for l in range(p.L):
        V = sum(p.lam * x[i, l] * n_op[i] for i in range(N))
        P = scipy.linalg.expm(-p.dtau * V) @ eK @ P
    Z1 = np.trace(P)
    lndet, sign, G = fermion_logdet(p, x)
    assert abs(np.log(abs(Z1)) - lndet) < 1e-11 and np.sign(Z1) == sign
    Gf = np.array([[np.trace(c[i] @ c[j].T @ P) / Z1 for j in range(N)] for i in range(N)])
    assert np.abs(Gf - G).max() < 1e-12
    # Two identical independent spin species: <n_i n_j> = 2<n_i n_j>_s + 2<n_i>_s <n_j>_s
    nn1 = np.array([[np.trace(n_op[i] @ n_op[j] @ P) / Z1 for j in range(N)] for i in range(N)])
    n1 = np.array([np.trace(n_op[i] @ P) / Z1 for i in range(N)])
    nn = 2 * nn1 + 2 * np.outer(n1, n1)
    s = staggered_sign(2, 2)
    assert abs(s @ nn @ s / N - s_cdw(p, G)) < 1e-12


def test_free_fermion_structure_factor():
    # lam = 0: S = 1 - (2/N) sum_k f_k (1 - f_k), f_k = 1/(1 + e^{-beta eps_k}).
    for Lx, L in ((4, 40), (6, 30)):
        p = HolsteinParams(Lx, Lx, L, lam=0.0, n_s=10)
        _, _, G = fermion_logdet(p, np.zeros((p.N, L)))
        eps, _, _ = dispersion(Lx, Lx, 1.0, 0.0)
        f = 1 / (1 + np.exp(-p.beta * eps))
        assert abs(s_cdw(p, G) - (1 - 2 / p.N * np.sum(f * (1 - f)))) < 1e-12


def test_atomic_limit_structure_factor_by_enumeration():
    # t = 0: sites and spins independent; enumerate all 2^(2N) occupations of a 2x2 lattice.
    p = HolsteinParams(2, 2, 5, t=0.0, lam=1.0, n_s=5)
    x = np.random.default_rng(3).normal(size=(4, 5))
    _, _, G = fermion_logdet(p, x)
    h = p.dtau * p.lam * x.sum(axis=1)  # each electron on site i gets weight e^{-h_i}
    s = staggered_sign(2, 2)
    Z = 0.0
    acc = 0.0
    for occ in itertools.product((0, 1), repeat=8):
        n = np.array(occ[:4]) + np.array(occ[4:])
        wgt = np.exp(-np.sum(h * n))
        Z += wgt
        acc += wgt * (s @ n) ** 2
    assert abs(acc / Z / 4 - s_cdw(p, G)) < 1e-12
