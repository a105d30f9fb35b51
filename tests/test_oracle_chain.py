"""Pins of the oracle's effective-model sweeps and cumulative update (Eq. (6)):
sequential equivalence of checkerboard half-sweeps, exact sampling of Gaussian and
decoupled double-well models, acceptance 1 when E_eff equals the exact weight, and
independence of the sampled distribution from the choice of E_eff."""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import HolsteinParams
from oracle.chain import colour_mask, cumulative_update, eff_sweeps, half_sweep, update_draws
from oracle.effective import local_energy, log_weight_eff
from oracle.lattice import exp_hopping
from oracle.philox import philox4x32_10, seed_key, uniform53
from oracle.weight import log_weight


def test_half_sweep_equals_sequential_metropolis():
    p = HolsteinParams(4, 2, 4, lam=0.8)
    J = np.array([20.0, 0.5, 0.02, 0.3, -0.2])
    rng = np.random.default_rng(0)
    x0 = rng.normal(size=(p.N, p.L))
    for colour in (0, 1):
        xv = x0.copy()
        nv = half_sweep(p, xv, J, colour, 17, 3, 99, 0.7)
        xs = x0.copy()
        ns = 0
        for i in range(p.N):
            for l in range(p.L):
                if ((i % p.Lx) + (i // p.Lx) + l) % 2 != colour:
                    continue
                w = philox4x32_10((i * p.L + l, 17, 3, 0), seed_key(99))
                xn = xs[i, l] + 0.7 * (2 * uniform53(w[0], w[1]) - 1)
                ix, iy = i % p.Lx, i // p.Lx
                nb = sum(xs[((ix + dx) % p.Lx) + p.Lx * ((iy + dy) % p.Ly), l]
                         for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)))
                up, dn = xs[i, (l + 1) % p.L], xs[i, (l - 1) % p.L]
                dE = local_energy(p, J, xn, up, dn, nb) - local_energy(p, J, xs[i, l], up, dn, nb)
                if -p.dtau * dE >= 0 or uniform53(w[2], w[3]) < math.exp(-p.dtau * dE):
                    xs[i, l] = xn
                    ns += 1
        assert nv == ns
        assert np.array_equal(xv, xs)


def _batch_error(samples, nbins=20):
    b = np.array_split(np.asarray(samples), nbins)
    m = np.array([np.mean(v, axis=0) for v in b])
    return np.std(m, axis=0, ddof=1) / math.sqrt(nbins)


@pytest.mark.slow
def test_sweeps_sample_gaussian_model_exactly():
    # J_p = J_p' = 0: ln w_eff = -dtau x^T A x, covariance (2 dtau A)^-1, with A built from
    # explicit bond lists (not from the oracle's features).
    Lx, Ly, L = 4, 4, 4
    p = HolsteinParams(Lx, Ly, L)
    Jk, Jnn, Jnnp = 5.0, 0.5, 4.0
    n = Lx * Ly * L
    q = lambda i, l: i * L + l
    A = np.zeros((n, n))
    for iy in range(Ly):
        for ix in range(Lx):
            i = ix + Lx * iy
            for l in range(L):
                d = np.zeros(n)
                d[q(i, (l + 1) % L)] += 1
                d[q(i, l)] -= 1
                A += Jk * np.outer(d, d)
                a, b = q(i, l), q(i, (l + 1) % L)
                A[a, b] += Jnnp / 2
                A[b, a] += Jnnp / 2
                for j in (((ix + 1) % Lx) + Lx * iy, ix + Lx * ((iy + 1) % Ly)):
                    a, b = q(i, l), q(j, l)
                    A[a, b] += Jnn / 2
                    A[b, a] += Jnn / 2
    C = np.linalg.inv(2 * p.dtau * A)
    J = np.array([Jk, 0.0, 0.0, Jnn, Jnnp])
    x = np.zeros((p.N, L))
    obs = []
    for s in range(12000):
        eff_sweeps(p, x, J, 1, s, s % 2, 0, 12345, 1.6)
        if s >= 500:
            # translation-averaged <x_0 x_r> for r in {same site, +l, +x, +x+l}
            o = [np.mean(x * x), np.mean(x * np.roll(x, -1, axis=1)),
                 np.mean(x.reshape(Ly, Lx, L) * np.roll(x.reshape(Ly, Lx, L), -1, axis=1)),
                 np.mean(x.reshape(Ly, Lx, L) * np.roll(np.roll(x.reshape(Ly, Lx, L), -1, axis=1), -1, axis=2))]
            obs.append(o)
    mean = np.mean(obs, axis=0)
    err = _batch_error(obs)
    ref = [C[0, 0], C[q(0, 0), q(0, 1)], C[q(0, 0), q(1, 0)], C[q(0, 0), q(1, 1)]]
    assert np.all(np.abs(mean - ref) < 5 * err + 1e-3), (mean, ref, err)


@pytest.mark.slow
def test_sweeps_sample_decoupled_double_well():
    p = HolsteinParams(4, 4, 4, lam=1.0)
    Jp, Jpp = 30.0, 4.0
    J = np.array([0.0, Jp, Jpp, 0.0, 0.0])
    a2 = p.a ** 2
    w = lambda v: math.exp(-p.dtau * (Jp * (v ** 4 / 4 - a2 * v ** 2 / 2) + Jpp * (v ** 6 / 6 - a2 * v ** 4 / 4)))
    Z = scipy.integrate.quad(w, -6, 6, points=[-1, 0, 1])[0]
    m2 = scipy.integrate.quad(lambda v: v * v * w(v), -6, 6, points=[-1, 0, 1])[0] / Z
    m4 = scipy.integrate.quad(lambda v: v ** 4 * w(v), -6, 6, points=[-1, 0, 1])[0] / Z
    x = np.zeros((p.N, p.L))
    obs = []
    for s in range(6000):
        eff_sweeps(p, x, J, 1, s, 0, 1, 777, 1.5)
        if s >= 200:
            obs.append([np.mean(x ** 2), np.mean(x ** 4)])
    mean = np.mean(obs, axis=0)
    err = _batch_error(obs)
    assert np.all(np.abs(mean - [m2, m4]) < 5 * err), (mean, [m2, m4], err)


def test_cumulative_update_accepts_everything_when_eff_is_exact():
    p = HolsteinParams(4, 4, 20, lam=0.0, n_s=10)
    E = exp_hopping(4, 4, 1.0, 0.0, 0.1)
    J = np.array([p.omega0 ** 2 / 4 + 1 / (2 * p.dtau ** 2), 0.0, 0.0, 0.0, p.omega0 ** 2 / 2])
    x = np.random.default_rng(1).normal(size=(16, 20))
    lnw = log_weight(p, x, E)[0]
    for u in range(15):
        x_before = x.copy()
        acc, lnw_new, G, nsw = cumulative_update(p, x, lnw, 0.0, J, 3, u, 0, 2024, 0.3, E=E)
        lnA = (lnw_new - lnw) - (log_weight_eff(p, x, 0.0, J) - log_weight_eff(p, x_before, 0.0, J))
        assert acc and abs(lnA) < 1e-9
        assert nsw > 0 and not np.array_equal(x, x_before)
        lnw = lnw_new


def test_update_draws_cover_both_colours():
    cols = [update_draws(u, 0, 5)[0] for u in range(64)]
    assert 10 < sum(cols) < 54


@pytest.mark.slow
def test_cumulative_update_samples_exact_weight_for_any_eff():
    # Eq. (6) makes the chain sample w, whatever E_eff proposes: two chains with very
    # different couplings must agree on <sum x^2> and on <x_i x_{i+x}> within errors.
    p = HolsteinParams(2, 2, 4, lam=1.0, n_s=2, dtau=0.25)
    E = exp_hopping(2, 2, 1.0, 0.0, p.dtau)
    results = []
    for J, delta in ((np.array([8.0, 0.5, 0.0, 0.0, 0.4]), 0.9),
                     (np.array([4.0, 0.0, 0.2, 0.2, 0.0]), 0.8)):
        x = np.zeros((4, 4))
        lnw = log_weight(p, x, E)[0]
        obs = []
        for u in range(3000):
            _, lnw, _, _ = cumulative_update(p, x, lnw, 0.0, J, 2, u, 0, 31337, delta, E=E)
            if u >= 100:
                obs.append([np.mean(x * x), np.mean(x * x[[1, 0, 3, 2], :])])
        results.append((np.mean(obs, axis=0), _batch_error(obs, 15)))
    (m1, e1), (m2, e2) = results
    assert np.all(np.abs(m1 - m2) < 4.5 * np.sqrt(e1 ** 2 + e2 ** 2)), results
