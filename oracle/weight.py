"""Full log-weight ln w(x) of a phonon configuration (oracle; test infrastructure only).

Sec. "Model" and Eq. (S2): w[X] = exp(-dtau S_Bose) (det M)^2 with
S_Bose = sum_{i,l} [Omega^2/2 X_il^2 + (X_{i,l+1} - X_il)^2 / dtau^2 * (1/2)].
Reading taken: the kinetic term carries the factor 1/2 of P^2/(2M) in Eq. (2) (the
printed sum omits it); Table S1's J_k = 50.0 = 1/(2 dtau^2) at dtau = 0.1 is the bare
coefficient with that 1/2. With the particle-hole symmetric coupling lam x (n - 1),
each spin species also contributes exp(+dtau lam x / 2) per site and slice, so
    ln w = 2 ln|det M| + dtau lam sum x - dtau sum [omega0^2 x^2 / 2 + (x_{l+1} - x_l)^2 / (2 dtau^2)]
with l periodic. Sums are exactly rounded (math.fsum).
"""
import math

import numpy as np

from .fermion import fermion_logdet


def bose_log_weight(p, x):
    """dtau lam sum x - dtau S_Bose (everything in ln w except 2 ln|det M|)."""
    x = np.asarray(x, dtype=np.float64)
    dx = np.roll(x, -1, axis=1) - x
    terms = (p.dtau * p.lam * x
             - p.dtau * (0.5 * p.omega0 ** 2 * x * x + dx * dx / (2.0 * p.dtau ** 2)))
    return math.fsum(terms.ravel().tolist())


def log_weight(p, x, E=None):
    """(ln w, ln|det M|, sign, G)."""
    lndet, sign, G = fermion_logdet(p, x, E=E)
    return 2.0 * lndet + bose_log_weight(p, x), lndet, sign, G
