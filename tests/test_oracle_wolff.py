"""Pins of the oracle's modified Wolff cluster update of E_eff (Sec. "Wolff update of the
effective Hamiltonian", Eq. (S9)): exact detailed balance of the cluster move with respect to
w_eff, by enumerating every bond-activation pattern and seed on small lattices; the Ising limit
of the activation probability; invariance of every E_eff term but F_nn, whose change is
carried by the cluster boundary alone; and the composite sweep order."""
import itertools
import math

import numpy as np
import pytest

from oracle import HolsteinParams
from oracle.chain import eff_sweeps, wolff_activation_prob, wolff_bonds, wolff_cluster, wolff_update
from oracle.effective import features, log_weight_eff


def _cluster_probabilities(p, x, J):
    """T(x -> x with the columns of C reflected) for every cluster C, by enumeration of all
    activation patterns of the 2N bond terms and all seed sites."""
    _, padd = wolff_activation_prob(p, x, J)
    nb = 2 * p.N
    out = {}
    for pattern in itertools.product((False, True), repeat=nb):
        act = np.array(pattern)
        prob = float(np.prod(np.where(act, padd, 1.0 - padd)))
        if prob == 0.0:
            continue
        for seed in range(p.N):
            c = wolff_cluster(p, act, seed)
            key = tuple(np.nonzero(c)[0])
            out[key] = out.get(key, 0.0) + prob / p.N
    return out


@pytest.mark.parametrize("Lx,Ly,L,Jnn", [(2, 2, 2, 0.9), (2, 2, 3, -0.7), (3, 2, 2, 1.3)])
def test_detailed_balance_by_enumeration(Lx, Ly, L, Jnn):
    p = HolsteinParams(Lx, Ly, L, lam=1.1, omega0=0.8)
    J = np.array([30.0, 0.4, 0.03, Jnn, 0.2])
    rng = np.random.default_rng(Lx * 10 + L)
    x = rng.normal(scale=1.5, size=(p.N, p.L))
    forward = _cluster_probabilities(p, x, J)
    assert abs(sum(forward.values()) - 1.0) < 1e-12
    for cl, t_fwd in forward.items():
        xr = x.copy()
        xr[list(cl)] = -xr[list(cl)]
        t_back = _cluster_probabilities(p, xr, J).get(cl, 0.0)
        lhs = t_fwd * math.exp(log_weight_eff(p, x, 0.0, J))
        rhs = t_back * math.exp(log_weight_eff(p, xr, 0.0, J))
        assert abs(lhs - rhs) <= 1e-10 * max(lhs, rhs), (cl, t_fwd, t_back)


def test_ising_limit():
    """Columns x_il = sigma_i (constant in time): the bond term is an Ising bond of strength
    dtau J_nn L, and P_add is the textbook 1 - exp(-2 beta |J|) for bonds that reflecting one
    end would weaken (anti-aligned for J_nn > 0), 0 for the others."""
    p = HolsteinParams(4, 4, 6)
    rng = np.random.default_rng(3)
    sigma = rng.choice([-1.0, 1.0], size=p.N)
    x = np.repeat(sigma[:, None], p.L, axis=1)
    for Jnn in (0.35, -0.35):
        J = np.array([50.0, 0.0, 0.0, Jnn, 0.0])
        _, padd = wolff_activation_prob(p, x, J)
        bi, bj = wolff_bonds(p)
        weakened = Jnn * sigma[bi] * sigma[bj] < 0
        expected = np.where(weakened, 1.0 - math.exp(-2.0 * p.dtau * abs(Jnn) * p.L), 0.0)
        assert np.allclose(padd, expected, rtol=1e-14, atol=0.0)


def test_move_changes_only_the_boundary_bonds():
    p = HolsteinParams(6, 4, 8, lam=1.0)
    J = np.array([50.0, 0.1, 0.0, 0.6, 0.3])
    rng = np.random.default_rng(11)
    bi, bj = wolff_bonds(p)
    sizes = []
    for ctr in range(40):
        x = rng.normal(size=(p.N, p.L))
        x0 = x.copy()
        n = wolff_update(p, x, J, ctr, 5, 12345)
        sizes.append(n)
        flipped = np.all(x == -x0, axis=1) & np.any(x0 != 0, axis=1)
        assert flipped.sum() == n and np.all((x == x0)[~flipped])
        f0, f1 = features(p, x0), features(p, x)
        for q in (0, 1, 2, 4):  # F_k, F_p, F_p', F_nn': invariant under reflecting whole columns
            assert abs(f1[q] - f0[q]) <= 1e-11 * max(1.0, abs(f0[q]))
        boundary = flipped[bi] != flipped[bj]
        s = np.einsum("bl,bl->b", x0[bi], x0[bj])
        assert abs((f1[3] - f0[3]) - (-2.0 * s[boundary].sum())) <= 1e-10 * max(1.0, abs(f0[3]))
        # no activated bond crosses the boundary: its probability from the old state is 0 or
        # the bond was not drawn; bonds with P_add = 1 - exp(t) ~ 1 must then lie inside
        _, padd = wolff_activation_prob(p, x0, J)
        assert np.all(padd[boundary] < 1.0)
    assert 1 <= min(sizes) and max(sizes) <= p.N and len(set(sizes)) > 3


def test_sweeps_with_wolff_are_the_old_sweeps_without_it():
    p = HolsteinParams(4, 4, 6)
    J = np.array([50.0, 0.2, 0.0, 0.5, 0.3])
    rng = np.random.default_rng(2)
    x = rng.normal(size=(p.N, p.L))
    a, b = x.copy(), x.copy()
    eff_sweeps(p, a, J, 3, 7, 1, 2, 99, 0.4)
    sizes = []
    eff_sweeps(p, b, J, 3, 7, 1, 2, 99, 0.4, nwolff=0, wolff_sizes=sizes)
    assert np.array_equal(a, b) and sizes == []
    c = x.copy()
    eff_sweeps(p, c, J, 3, 7, 1, 2, 99, 0.4, nwolff=2, wolff_sizes=sizes)
    assert len(sizes) == 6 and not np.array_equal(a, c)
