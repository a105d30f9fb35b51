"""Conventional DQMC updates of the phonon field (oracle; test infrastructure only).

Supplemental Material, Sec. "DQMC for the Holstein model", Eqs. (S3)-(S6), and the block
update described after them:
  * local update of x_{i,l-1} (the field of B_l) at time slice l: per spin species the
    fermion ratio is R = 1 + (1 - G_ii(l)) Delta_ii with Delta_ii = exp(-dtau lam d) - 1,
    d the change of the field (Eq. (S5)); both species are equal, so the weight ratio is
    R^2 exp(d ln w_bose); an accepted move updates G(l) by Sherman-Morrison (Eq. (S6));
  * G is carried from slice l - 1 to slice l by G(l) = B_l G(l-1) B_l^-1 (from the
    definition of G(l), Eq. (S3)) and recomputed from scratch at the start of every group
    of n_s slices (the paper gives no stabilisation interval; n_s is reused);
  * block update: the field of one site is reflected on every slice about the mirror axis
    (x -> -x in the shifted field; the paper's X -> -X - 2g/Omega^2), accepted with the
    ratio of the full weights.
Readings where the paper is silent: the local proposal is x' = x + U[-Delta, Delta] (as
for the effective model); slices are visited in order 1..L and the sites of a slice in
order i = 0..N-1; random numbers come from Philox-4x32-10 with key = seed, counter
(i L + l - 1, sweep, chain, 3) for the local move at (i, l) (words 0-1: proposal,
2-3: acceptance) and (k, sweep, chain, 4) for block update k (words 0-1: site,
2-3: acceptance).
"""
import math

import numpy as np

from .fermion import fermion_logdet, slice_scales
from .lattice import exp_hopping
from .philox import philox4x32_10, seed_key, uniform53
from .weight import log_weight


def greens_at(p, x, l, E):
    """G(l) = [I + B_l ... B_1 B_L ... B_{l+1}]^-1 (Eq. (S3)): the equal-time Green's function
    G(L) of the field rotated by l slices (column l of x becomes the field of B_1)."""
    return fermion_logdet(p, np.roll(x, -l, axis=1), E)[2]


def wrap(p, G, x_col, E, Einv):
    """G(l) = B_l G(l-1) B_l^-1 with B_l = diag(s) E, s = exp(-dtau lam x_{:, l-1})."""
    s = slice_scales(x_col, p.dtau, p.lam)
    return s[:, None] * (E @ (G @ Einv)) / s[None, :]


def bose_change(p, v, vn, up, dn):
    """Change of dtau lam sum x - dtau S_Bose when one site's field goes from v to vn,
    given its time neighbours up = x_{i,l+1} and dn = x_{i,l-1} (periodic)."""
    kin = ((up - vn) ** 2 + (vn - dn) ** 2 - (up - v) ** 2 - (v - dn) ** 2) / (2.0 * p.dtau ** 2)
    return p.dtau * p.lam * (vn - v) - p.dtau * (0.5 * p.omega0 ** 2 * (vn * vn - v * v) + kin)


def local_move(p, x, G, i, c, sweep, chain, seed, delta):
    """The proposal and log acceptance ratio of the local move at site i, field column c, given
    G = G(c + 1). Returns (xn, Delta_ii, R, ln ratio, u_acc)."""
    w = philox4x32_10((np.uint32(i * p.L + c), np.uint32(sweep), np.uint32(chain), np.uint32(3)), seed_key(seed))
    u1, u2 = float(uniform53(w[0], w[1])), float(uniform53(w[2], w[3]))
    v = x[i, c]
    xn = v + delta * (2.0 * u1 - 1.0)
    dl = math.exp(-p.dtau * p.lam * (xn - v)) - 1.0
    R = 1.0 + (1.0 - G[i, i]) * dl
    dlb = bose_change(p, v, xn, x[i, (c + 1) % p.L], x[i, (c - 1) % p.L])
    lnr = math.log(R * R) + dlb if R != 0.0 else -math.inf
    return xn, dl, R, lnr, u2


def sherman_morrison(G, i, dl, R):
    """G' = G - G Delta (I - G) / R for Delta = dl e_i e_i^T (Eq. (S6))."""
    row = -G[i, :].copy()
    row[i] += 1.0
    return G - (dl / R) * np.outer(G[:, i], row)


def local_sweep(p, x, sweep, chain, seed, delta, E=None, Einv=None):
    """One sweep of local updates over all slices and sites, in place; returns #accepted."""
    if E is None:
        E = exp_hopping(p.Lx, p.Ly, p.t, p.mu, p.dtau)
    if Einv is None:
        Einv = exp_hopping(p.Lx, p.Ly, p.t, p.mu, -p.dtau)
    n_acc = 0
    for g0 in range(0, p.L, p.n_s):
        G = greens_at(p, x, g0, E)
        for l in range(g0 + 1, min(g0 + p.n_s, p.L) + 1):
            c = l - 1
            G = wrap(p, G, x[:, c], E, Einv)
            for i in range(p.N):
                xn, dl, R, lnr, u = local_move(p, x, G, i, c, sweep, chain, seed, delta)
                if lnr >= 0.0 or u < math.exp(lnr):
                    x[i, c] = xn
                    G = sherman_morrison(G, i, dl, R)
                    n_acc += 1
    return n_acc


def block_updates(p, x, nblock, sweep, chain, seed, E=None):
    """nblock block updates (reflection of one site's whole column), in place; returns
    #accepted."""
    n_acc = 0
    lnw = log_weight(p, x, E)[0]
    for k in range(nblock):
        w = philox4x32_10((np.uint32(k), np.uint32(sweep), np.uint32(chain), np.uint32(4)), seed_key(seed))
        site = min(p.N - 1, int(float(uniform53(w[0], w[1])) * p.N))
        u = float(uniform53(w[2], w[3]))
        xp = x.copy()
        xp[site] = -xp[site]
        lnw_new = log_weight(p, xp, E)[0]
        lnA = lnw_new - lnw
        if lnA >= 0.0 or u < math.exp(lnA):
            x[...] = xp
            lnw = lnw_new
            n_acc += 1
    return n_acc


def dqmc_sweeps(p, x, nsweeps, sweep0, chain, seed, delta, nblock=0, E=None):
    """nsweeps DQMC sweeps (local updates, then nblock block updates), sweep counters
    sweep0 .. sweep0 + nsweeps - 1; in place; returns (#local accepted, #block accepted)."""
    if E is None:
        E = exp_hopping(p.Lx, p.Ly, p.t, p.mu, p.dtau)
    Einv = exp_hopping(p.Lx, p.Ly, p.t, p.mu, -p.dtau)
    nl = nb = 0
    for s in range(nsweeps):
        nl += local_sweep(p, x, sweep0 + s, chain, seed, delta, E, Einv)
        nb += block_updates(p, x, nblock, sweep0 + s, chain, seed, E)
    return nl, nb
