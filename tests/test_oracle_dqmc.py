"""Pins of the oracle's conventional DQMC updates (Supplemental Material, Eqs. (S3)-(S6)):
the fast ratio R = 1 + (1 - G_ii) Delta_ii equals the ratio of the determinants computed from
scratch, the log acceptance ratio of a local move equals the difference of the full log-weights,
the Sherman-Morrison update equals G recomputed for the new field, and wrapping
G(l) = B_l G(l-1) B_l^-1 equals G(l) recomputed. Together with the symmetric proposal these
make the local sweep an exact Metropolis sampler of w."""
import math

import numpy as np
import pytest

from oracle import HolsteinParams
from oracle.dqmc import block_updates, dqmc_sweeps, greens_at, local_move, sherman_morrison, wrap
from oracle.fermion import fermion_logdet
from oracle.lattice import exp_hopping
from oracle.weight import log_weight


def _setup(Lx, Ly, L, n_s, seed, lam=1.0):
    p = HolsteinParams(Lx, Ly, L, n_s=n_s, lam=lam)
    E = exp_hopping(Lx, Ly, 1.0, 0.0, p.dtau)
    Einv = exp_hopping(Lx, Ly, 1.0, 0.0, -p.dtau)
    x = np.random.default_rng(seed).normal(scale=0.8, size=(p.N, p.L))
    return p, E, Einv, x


@pytest.mark.parametrize("Lx,Ly,L,n_s", [(4, 4, 12, 4), (3, 2, 6, 6), (2, 2, 2, 1)])
def test_fast_ratio_and_log_ratio_are_exact(Lx, Ly, L, n_s):
    p, E, _, x = _setup(Lx, Ly, L, n_s, Lx * 100 + L)
    ld, sg, _ = fermion_logdet(p, x, E)
    lw = log_weight(p, x, E)[0]
    for (i, c) in [(0, 0), (p.N - 1, L - 1), (1 % p.N, L // 2)]:
        G = greens_at(p, x, c + 1, E)
        xn, dl, R, lnr, _ = local_move(p, x, G, i, c, 5, 2, 99, 0.9)
        xp = x.copy()
        xp[i, c] = xn
        ld2, sg2, _ = fermion_logdet(p, xp, E)
        R_brute = sg * sg2 * math.exp(ld2 - ld)
        assert abs(R - R_brute) <= 1e-9 * abs(R_brute), (R, R_brute)
        assert abs(lnr - (log_weight(p, xp, E)[0] - lw)) <= 1e-8 * max(1.0, abs(lnr))


@pytest.mark.parametrize("Lx,Ly,L,n_s", [(4, 4, 12, 4), (3, 2, 6, 6)])
def test_sherman_morrison_and_wrap_equal_recomputation(Lx, Ly, L, n_s):
    p, E, Einv, x = _setup(Lx, Ly, L, n_s, 7)
    for (i, c) in [(0, 0), (p.N // 2, L - 1), (p.N - 1, 3)]:
        G = greens_at(p, x, c + 1, E)
        xn, dl, R, _, _ = local_move(p, x, G, i, c, 1, 0, 3, 1.2)
        Gn = sherman_morrison(G, i, dl, R)
        xp = x.copy()
        xp[i, c] = xn
        assert np.abs(Gn - greens_at(p, xp, c + 1, E)).max() < 1e-9
    for l in range(1, L + 1):
        Gw = wrap(p, greens_at(p, x, l - 1, E), x[:, l - 1], E, Einv)
        assert np.abs(Gw - greens_at(p, x, l, E)).max() < 1e-9


def test_sweeps_move_the_field_and_keep_it_finite():
    p, E, _, x = _setup(4, 4, 8, 4, 11)
    x0 = x.copy()
    nl, nb = dqmc_sweeps(p, x, 2, 10, 1, 123, 0.5, nblock=3, E=E)
    assert 0 < nl < 2 * p.N * p.L and 0 <= nb <= 6
    assert np.isfinite(x).all() and not np.array_equal(x, x0)


def test_block_update_reflects_whole_columns():
    p, E, _, x = _setup(4, 4, 8, 4, 12)
    x0 = x.copy()
    n = block_updates(p, x, 6, 3, 0, 77, E)
    changed = np.any(x != x0, axis=1)
    assert np.all(x[changed] == -x0[changed]) and changed.sum() <= n


@pytest.mark.parametrize("Lx,Ly,mu", [(4, 3, 0.3), (2, 5, 0.0), (6, 6, -0.2), (1, 4, 0.1)])
def test_hopping_exponential_factorises_into_circulants(Lx, Ly, mu):
    """exp(-dtau K) = e^{dtau mu} E_x kron E_y with E_x, E_y circulant one-dimensional factors (the
    x and y hoppings commute); the GPU wrap relies on it, and the mu factors of B and B^-1 cancel."""
    dtau, t = 0.1, 1.0

    def circ(Ld, a):
        k = 2.0 * np.pi * np.arange(Ld) / Ld
        d = np.subtract.outer(np.arange(Ld), np.arange(Ld)) % Ld
        return np.real(np.fft.ifft(np.exp(a * np.cos(k))))[d]

    E = exp_hopping(Lx, Ly, t, mu, dtau)
    # site i = ix + Lx iy: the y factor is the outer one of the Kronecker product
    assert np.abs(E - math.exp(dtau * mu) * np.kron(circ(Ly, 2 * dtau * t), circ(Lx, 2 * dtau * t))).max() < 1e-14
    Ei = exp_hopping(Lx, Ly, t, mu, -dtau)
    assert np.abs(Ei - math.exp(-dtau * mu) * np.kron(circ(Ly, -2 * dtau * t), circ(Lx, -2 * dtau * t))).max() < 1e-14
