"""Symmetric effective model E_eff and its linear-regression fit (oracle; test
infrastructure only).

Eq. (4) / Eq. (S7): -beta H_eff is a linear combination of five Z2-symmetric terms in
the shifted field x = X - alpha (alpha -> 0 with the particle-hole symmetric coupling,
alpha^2 -> a^2 = (lam/omega0^2)^2):
  F_k   = sum_{i,l} (x_{i,l+1} - x_il)^2                         (time, periodic)
  F_p   = sum_{i,l} (x^4/4 - a^2 x^2/2)                           (Fig. 1, blue)
  F_p'  = sum_{i,l} (x^6/6 - a^2 x^4/4)                           (Fig. 1, red)
  F_nn  = sum_{<ij>,l} x_il x_jl   (each periodic bond once: +x and +y from each site)
  F_nn' = sum_{i,l} x_il x_{i,l+1} (each time bond once, periodic)
Reading taken for sign and scale: ln w_eff = -dtau (E0 + J . F) with
J = (J_k, J_p, J_p', J_nn, J_nn'); the literal "-beta H_eff = +J_k ..." with J_k = +50
would not be normalisable, while J_k = 1/(2 dtau^2) is then exactly the bare phonon
kinetic coefficient (Table S1).
Eq. (5): the couplings are fitted by multi-linear least squares of ln w[x] on the
features; the constant E0 is the intercept.
"""
import math

import numpy as np

FEATURE_NAMES = ("F_k", "F_p", "F_p'", "F_nn", "F_nn'")


def features(p, x):
    """The five features of Eq. (S7) for x[N, L] (exactly rounded sums)."""
    x = np.asarray(x, dtype=np.float64)
    a2 = p.a ** 2
    X = x.reshape(p.Ly, p.Lx, p.L)               # [iy, ix, l]
    Xt = np.roll(X, -1, axis=2)                  # x_{i, l+1}
    Xx = np.roll(X, -1, axis=1)                  # x_{i + x^, l}
    Xy = np.roll(X, -1, axis=0)                  # x_{i + y^, l}
    x2 = X * X
    fs = lambda arr: math.fsum(arr.ravel().tolist())
    return np.array([
        fs((Xt - X) ** 2),
        fs(x2 * x2 / 4.0 - a2 * x2 / 2.0),
        fs(x2 * x2 * x2 / 6.0 - a2 * x2 * x2 / 4.0),
        fs(X * (Xx + Xy)),
        fs(X * Xt),
    ])


def log_weight_eff(p, x, E0, J):
    """ln w_eff = -dtau (E0 + J . F)."""
    F = features(p, x)
    return -p.dtau * (E0 + math.fsum((np.asarray(J) * F).tolist()))


def local_energy(p, J, v, x_up, x_dn, nbr_sum):
    """All terms of E0 + J . F that involve one site value v, given its two time
    neighbours x_up = x_{i,l+1}, x_dn = x_{i,l-1} and the sum of its four spatial
    neighbours. Differences of this for two values of v equal differences of the full
    E0 + J . F (pinned by a test)."""
    Jk, Jp, Jpp, Jnn, Jnnp = J
    a2 = p.a ** 2
    v2 = v * v
    return (Jk * ((x_up - v) ** 2 + (v - x_dn) ** 2)
            + Jp * (v2 * v2 / 4.0 - a2 * v2 / 2.0)
            + Jpp * (v2 * v2 * v2 / 6.0 - a2 * v2 * v2 / 4.0)
            + Jnn * v * nbr_sum
            + Jnnp * v * (x_up + x_dn))


def fit_couplings(p, xs, lnw):
    """Eq. (5): least squares of ln w on [1, F]; returns (E0, J[5], rms residual).
    numpy's SVD-based lstsq serves as the solver."""
    Phi = np.array([np.concatenate(([1.0], features(p, x))) for x in xs])
    y = np.asarray(lnw, dtype=np.float64)
    c, *_ = np.linalg.lstsq(Phi, y, rcond=None)
    resid = float(np.sqrt(np.mean((Phi @ c - y) ** 2)))
    coef = -c / p.dtau
    return float(coef[0]), coef[1:], resid
