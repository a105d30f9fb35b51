"""Effective-model Markov chain and the cumulative update with exact acceptance
(oracle; test infrastructure only).

Sec. "SLMC" and Sec. "Wolff update of the effective Hamiltonian" (last paragraph): the
proposal for the original model is built from local updates of the phonon field under
the cheap bosonic E_eff; Eq. (6) then accepts the final configuration with
    A = min{1, [w(x') / w(x)] [w_eff(x) / w_eff(x')]}.
Readings taken where the paper is silent:
  * local proposal x' = x + delta, delta uniform in [-Delta, Delta], Metropolis
    acceptance under w_eff;
  * sites are visited in checkerboard half-sweeps of colour (ix + iy + l) mod 2
    (same-colour sites share no term of E_eff, so a half-sweep equals any sequential
    order); one sweep = both colours;
  * the starting colour of every cumulative update is drawn with probability 1/2,
    which makes the composite proposal reversible with respect to w_eff, so Eq. (6)
    is exact;
  * random numbers follow the Philox layout documented in oracle.philox.
Sites of one colour are updated together with numpy (they are independent).
"""
import math

import numpy as np

from .effective import local_energy, log_weight_eff
from .lattice import coords
from .philox import philox4x32_10, seed_key, uniform53
from .weight import log_weight


def colour_mask(p, c):
    ix, iy = coords(p.N, p.Lx)
    l = np.arange(p.L)
    return ((ix[:, None] + iy[:, None] + l[None, :]) % 2) == c


def neighbour_sum(p, x):
    X = x.reshape(p.Ly, p.Lx, p.L)
    s = (np.roll(X, -1, axis=1) + np.roll(X, 1, axis=1)
         + np.roll(X, -1, axis=0) + np.roll(X, 1, axis=0))
    return s.reshape(p.N, p.L)


def half_sweep(p, x, J, colour, sweep, chain, seed, delta):
    """Metropolis update of every site of one colour, in place; returns #accepted."""
    N, L = p.N, p.L
    site_ctr = (np.arange(N)[:, None] * L + np.arange(L)[None, :]).astype(np.uint32)
    w = philox4x32_10((site_ctr, np.uint32(sweep), np.uint32(chain), np.uint32(0)), seed_key(seed))
    u_prop = uniform53(w[0], w[1])
    u_acc = uniform53(w[2], w[3])
    x_up = np.roll(x, -1, axis=1)
    x_dn = np.roll(x, 1, axis=1)
    nb = neighbour_sum(p, x)
    xn = x + delta * (2.0 * u_prop - 1.0)
    dE = local_energy(p, J, xn, x_up, x_dn, nb) - local_energy(p, J, x, x_up, x_dn, nb)
    dlnw = -p.dtau * dE
    with np.errstate(over="ignore"):
        acc = colour_mask(p, colour) & ((dlnw >= 0.0) | (u_acc < np.exp(dlnw)))
    x[acc] = xn[acc]
    return int(acc.sum())


def eff_sweeps(p, x, J, nsweeps, sweep0, first_colour, chain, seed, delta):
    """nsweeps full sweeps (colours first_colour, 1 - first_colour) with sweep
    counters sweep0 .. sweep0 + nsweeps - 1; in place; returns #accepted moves."""
    n_acc = 0
    for s in range(nsweeps):
        for c in (first_colour, 1 - first_colour):
            n_acc += half_sweep(p, x, J, c, sweep0 + s, chain, seed, delta)
    return n_acc


def update_draws(update, chain, seed):
    w = philox4x32_10((np.uint32(update), np.uint32(0), np.uint32(chain), np.uint32(1)), seed_key(seed))
    return int(w[0]) & 1, float(uniform53(w[2], w[3]))


def cumulative_update(p, x, lnw, E0, J, nsweeps, update, chain, seed, delta, E=None):
    """One cumulative update of Eq. (6) for one chain. x is modified in place (kept on
    acceptance, restored on rejection). lnw is the cached exact ln w(x).
    Returns (accepted, lnw_new_state, G_of_new_state_or_None, n_sweep_accepts)."""
    first, u = update_draws(update, chain, seed)
    x_old = x.copy()
    lnweff_old = log_weight_eff(p, x, E0, J)
    n_sw = eff_sweeps(p, x, J, nsweeps, update * nsweeps, first, chain, seed, delta)
    lnweff_new = log_weight_eff(p, x, E0, J)
    lnw_new, _, _, G = log_weight(p, x, E=E)
    lnA = (lnw_new - lnw) - (lnweff_new - lnweff_old)
    accepted = lnA >= 0.0 or u < math.exp(lnA)
    if accepted:
        return True, lnw_new, G, n_sw
    x[...] = x_old
    return False, lnw, None, n_sw
