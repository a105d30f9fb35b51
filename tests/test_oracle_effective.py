"""Pins of the oracle's effective model (Eq. (4)/(S7)) and regression fit (Eq. (5))."""
import json
import os

import numpy as np
import pytest

from oracle import HolsteinParams
from oracle.effective import features, fit_couplings, local_energy, log_weight_eff
from oracle.chain import neighbour_sum
from oracle.lattice import exp_hopping
from oracle.weight import log_weight

HERE = os.path.dirname(os.path.abspath(__file__))


def brute_features(Lx, Ly, L, a, x):
    """Explicit loops over sites, bonds (as a set of unordered pairs) and time bonds."""
    idx = lambda ix, iy: (ix % Lx) + Lx * (iy % Ly)
    bonds = set()
    for iy in range(Ly):
        for ix in range(Lx):
            for j in (idx(ix + 1, iy), idx(ix, iy + 1)):
                bonds.add(frozenset((idx(ix, iy), j)))
    Fk = Fp = Fpp = Fnn = Fnnp = 0.0
    for i in range(Lx * Ly):
        for l in range(L):
            v = x[i, l]
            w = x[i, (l + 1) % L]
            Fk += (w - v) ** 2
            Fp += v ** 4 / 4 - a * a * v * v / 2
            Fpp += v ** 6 / 6 - a * a * v ** 4 / 4
            Fnnp += v * w
    for b in bonds:
        i, j = tuple(b)
        for l in range(L):
            Fnn += x[i, l] * x[j, l]
    return np.array([Fk, Fp, Fpp, Fnn, Fnnp])


@pytest.mark.parametrize("Lx,Ly,L", [(3, 4, 3), (4, 4, 5), (5, 3, 4)])
def test_features_against_loops(Lx, Ly, L):
    p = HolsteinParams(Lx, Ly, L, lam=1.3, omega0=0.9)
    x = np.random.default_rng(Lx * Ly * L).normal(size=(p.N, L))
    assert np.allclose(features(p, x), brute_features(Lx, Ly, L, p.a, x), rtol=1e-13, atol=1e-12)


def test_z2_mirror_symmetry():
    p = HolsteinParams(4, 4, 8)
    x = np.random.default_rng(1).normal(size=(16, 8))
    J = np.array([50.0, 0.3, -0.01, 0.2, 0.5])
    assert abs(log_weight_eff(p, x, 1.0, J) - log_weight_eff(p, -x, 1.0, J)) < 1e-11


@pytest.mark.parametrize("Lx,Ly,L", [(4, 4, 6), (2, 2, 2), (2, 4, 2)])
def test_local_energy_difference_equals_full_difference(Lx, Ly, L):
    p = HolsteinParams(Lx, Ly, L, lam=1.1)
    rng = np.random.default_rng(2)
    J = np.array([50.0, 0.7, 0.05, 0.3, -0.4])
    x = rng.normal(size=(p.N, L))
    for _ in range(10):
        i, l = rng.integers(p.N), rng.integers(L)
        v = x[i, l] + rng.normal()
        y = x.copy()
        y[i, l] = v
        full = (log_weight_eff(p, y, 0.0, J) - log_weight_eff(p, x, 0.0, J)) / (-p.dtau)
        nb = neighbour_sum(p, x)[i, l]
        loc = (local_energy(p, J, v, x[i, (l + 1) % L], x[i, (l - 1) % L], nb)
               - local_energy(p, J, x[i, l], x[i, (l + 1) % L], x[i, (l - 1) % L], nb))
        assert abs(full - loc) < 1e-9 * max(1.0, abs(full))


def test_double_well_basis_minima():
    # Fig. 1: both basis functions have minima at +-|alpha| and a maximum at 0.
    a = 1.7
    xs = np.linspace(-3, 3, 600001)
    for f in (lambda x: x ** 4 / 4 - a * a * x ** 2 / 2, lambda x: x ** 6 / 6 - a * a * x ** 4 / 4):
        y = f(xs)
        neg, pos = xs < 0, xs > 0
        assert abs(xs[neg][np.argmin(y[neg])] + a) < 1e-4
        assert abs(xs[pos][np.argmin(y[pos])] - a) < 1e-4
        mid = np.abs(xs) < a / 2
        assert abs(xs[mid][np.argmax(y[mid])]) < 1e-4


def test_fit_recovers_known_couplings_exactly():
    p = HolsteinParams(4, 4, 10, lam=1.0)
    rng = np.random.default_rng(3)
    E0, J = 3.5, np.array([50.0, 0.12, -0.004, 0.07, 0.3])
    xs = [rng.normal(size=(16, 10)) * rng.uniform(0.5, 1.5) + rng.uniform(-0.3, 0.3) for _ in range(60)]
    ys = [log_weight_eff(p, x, E0, J) for x in xs]
    E0f, Jf, res = fit_couplings(p, xs, ys)
    assert abs(E0f - E0) < 1e-7 * 50 and np.allclose(Jf, J, rtol=1e-7, atol=1e-9)
    assert res < 1e-8


def test_fit_lambda_zero_is_exact_bare_action():
    # At lam = 0 the determinant is field independent and sum x^2 = (F_k + 2 F_nn')/2, so
    # ln w = const - dtau [(omega0^2/4 + 1/(2 dtau^2)) F_k + (omega0^2/2) F_nn'] exactly.
    p = HolsteinParams(4, 4, 20, lam=0.0, omega0=1.0, n_s=10)
    E = exp_hopping(4, 4, 1.0, 0.0, 0.1)
    rng = np.random.default_rng(4)
    xs = [rng.normal(size=(16, 20)) * rng.uniform(0.5, 1.5) for _ in range(30)]
    ys = [log_weight(p, x, E)[0] for x in xs]
    E0f, Jf, res = fit_couplings(p, xs, ys)
    ref = np.array([0.25 + 50.0, 0.0, 0.0, 0.0, 0.5])
    assert np.allclose(Jf, ref, atol=1e-7)


def test_table_s1_kinetic_coupling():
    # Fitting the exact ln w of the oracle reproduces Table S1's J_k = 50.0 = 1/(2 dtau^2)
    # (to ~1 %), which pins the 1/2 of the phonon kinetic term and the reading
    # ln w_eff = -dtau (E0 + J . F).
    gold = json.load(open(os.path.join(HERE, "golden", "table_s1.json")))
    p = HolsteinParams(4, 4, 40, n_s=10)
    E = exp_hopping(4, 4, 1.0, 0.0, p.dtau)
    rng = np.random.default_rng(5)
    xs = [rng.normal(size=(16, 40)) * rng.uniform(0.3, 1.5) for _ in range(120)]
    ys = [log_weight(p, x, E)[0] for x in xs]
    _, Jf, _ = fit_couplings(p, xs, ys)
    assert abs(Jf[0] - gold["J_k"]) < 0.01 * gold["J_k"]
    assert abs(gold["J_k"] - 1.0 / (2 * gold["dtau"] ** 2)) < 1e-12
