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
  * random numbers follow the Philox layout documented in oracle.philox;
  * the optional modified Wolff cluster updates (Sec. "Wolff update of the effective
    Hamiltonian", Eq. (S9)) run between the two half-sweeps of every sweep, so the
    reversed sequence of a cumulative update is the sequence with the other starting
    colour and the composite proposal stays reversible.
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


def eff_sweeps(p, x, J, nsweeps, sweep0, first_colour, chain, seed, delta, nwolff=0, wolff_sizes=None):
    """nsweeps full sweeps (colours first_colour, 1 - first_colour) with sweep
    counters sweep0 .. sweep0 + nsweeps - 1, and nwolff Wolff updates between the two
    colours of every sweep (counters (sweep counter) * nwolff + k, mod 2^32); in place;
    returns #accepted local moves (cluster sizes are appended to wolff_sizes)."""
    n_acc = 0
    for s in range(nsweeps):
        n_acc += half_sweep(p, x, J, first_colour, sweep0 + s, chain, seed, delta)
        for k in range(nwolff):
            n = wolff_update(p, x, J, ((sweep0 + s) * nwolff + k) & 0xFFFFFFFF, chain, seed)
            if wolff_sizes is not None:
                wolff_sizes.append(n)
        n_acc += half_sweep(p, x, J, 1 - first_colour, sweep0 + s, chain, seed, delta)
    return n_acc


def wolff_bonds(p):
    """The 2N spatial bond terms of F_nn: b = 2 i is (i, i + x^), b = 2 i + 1 is (i, i + y^)."""
    ix, iy = coords(p.N, p.Lx)
    jx = (ix + 1) % p.Lx + p.Lx * iy
    jy = ix + p.Lx * ((iy + 1) % p.Ly)
    bi = np.repeat(np.arange(p.N), 2)
    bj = np.stack([jx, jy], axis=1).reshape(-1)
    return bi, bj


def wolff_activation_prob(p, x, J):
    """Probability of activating each bond term b = (i, j) of J_nn F_nn [Eq. (S9)].
    The term contributes exp(-dtau J_nn s_b), s_b = sum_l x_il x_jl, to w_eff; reflecting the
    whole column of one endpoint (x -> -x, the mirror about the symmetry axis) turns it into
    exp(+dtau J_nn s_b). Following the embedded-cluster construction, the bond is activated
    with probability max(0, 1 - exp(2 dtau J_nn s_b)). s_b is summed over l in order (the
    order the GPU uses, so that both take the same floating-point decisions).
    Returns (t_b = 2 dtau J_nn s_b, P_add)."""
    bi, bj = wolff_bonds(p)
    s = np.cumsum(x[bi] * x[bj], axis=1)[:, -1]
    t = (2.0 * p.dtau * J[3]) * s
    with np.errstate(over="ignore"):
        padd = np.where(t < 0.0, 1.0 - np.exp(np.minimum(t, 0.0)), 0.0)
    return t, padd


def wolff_cluster(p, active, seed_site):
    """Sites connected to seed_site through the activated bond terms (boolean [N])."""
    bi, bj = wolff_bonds(p)
    nbrs = [[] for _ in range(p.N)]
    for b in np.nonzero(active)[0]:
        nbrs[bi[b]].append(bj[b])
        nbrs[bj[b]].append(bi[b])
    in_c = np.zeros(p.N, dtype=bool)
    in_c[seed_site] = True
    stack = [seed_site]
    while stack:
        i = stack.pop()
        for j in nbrs[i]:
            if not in_c[j]:
                in_c[j] = True
                stack.append(j)
    return in_c


def wolff_update(p, x, J, ctr, chain, seed):
    """One modified Wolff cluster update of E_eff (Sec. "Wolff update of the effective
    Hamiltonian", Eq. (S9)), in place; returns the number of reflected columns.
    The cluster is built in the spatial plane and includes whole temporal columns: each bond
    term is activated with the probability of wolff_activation_prob (uniform of Philox
    counter (b, ctr, chain, 2)), a seed site is drawn uniformly (counter (2N, ctr, chain, 2)),
    and every column of the seed's connected component is reflected. All other terms of
    E_eff are invariant under reflecting whole columns, so the move needs no acceptance step."""
    N = p.N
    t, _ = wolff_activation_prob(p, x, J)
    w = philox4x32_10((np.arange(2 * N + 1, dtype=np.uint32), np.uint32(ctr), np.uint32(chain), np.uint32(2)),
                      seed_key(seed))
    u = uniform53(w[0], w[1])
    with np.errstate(over="ignore"):
        active = (t < 0.0) & (u[:2 * N] < 1.0 - np.exp(np.minimum(t, 0.0)))
    seed_site = min(N - 1, int(u[2 * N] * N))
    in_c = wolff_cluster(p, active, seed_site)
    x[in_c] = -x[in_c]
    return int(in_c.sum())


def update_draws(update, chain, seed):
    w = philox4x32_10((np.uint32(update), np.uint32(0), np.uint32(chain), np.uint32(1)), seed_key(seed))
    return int(w[0]) & 1, float(uniform53(w[2], w[3]))


def cumulative_update(p, x, lnw, E0, J, nsweeps, update, chain, seed, delta, E=None, nwolff=0):
    """One cumulative update of Eq. (6) for one chain. x is modified in place (kept on
    acceptance, restored on rejection). lnw is the cached exact ln w(x).
    Returns (accepted, lnw_new_state, G_of_new_state_or_None, n_sweep_accepts)."""
    first, u = update_draws(update, chain, seed)
    x_old = x.copy()
    lnweff_old = log_weight_eff(p, x, E0, J)
    n_sw = eff_sweeps(p, x, J, nsweeps, update * nsweeps, first, chain, seed, delta, nwolff=nwolff)
    lnweff_new = log_weight_eff(p, x, E0, J)
    lnw_new, _, _, G = log_weight(p, x, E=E)
    lnA = (lnw_new - lnw) - (lnweff_new - lnweff_old)
    accepted = lnA >= 0.0 or u < math.exp(lnA)
    if accepted:
        return True, lnw_new, G, n_sw
    x[...] = x_old
    return False, lnw, None, n_sw
