"""Fermion determinant det(I + B_L ... B_1) and equal-time Green's function (oracle;
test infrastructure only).

Supplemental Material, Sec. "DQMC for the Holstein model":
  Eq. (S2): M = I + B_L B_{L-1} ... B_1 with B_l = exp(-dtau g X(l)) exp(-dtau K),
            identical for both spin species, so the weight carries (det M)^2.
  Eq. (S3): G(l) = [I + B_l ... B_1 B_L ... B_{l+1}]^(-1); the equal-time G returned
            here is G(L) = M^(-1).
With the particle-hole symmetric coupling, B_l = diag(exp(-dtau lam x[:, l])) E, E =
exp(-dtau K); column l-1 of x (0-based) belongs to B_l.

The paper gives no stabilisation scheme (it defers to the DQMC literature). The oracle
evaluates the plain product with the textbook UDT chain: every n_s slices the running
product B...B U D T is re-factored by a Householder QR with column pivoting (LAPACK's
geqp3 through scipy serves as the step), D = |diag R|, T <- D^-1 R P^T T, U <- Q; the
final determinant and inverse use the split D = D_b D_s (D_b = max(D,1), D_s = min(D,1))
so that M = U D_b (D_b^-1 U^T + D_s T). All arithmetic is FP64.
"""
import numpy as np
import scipy.linalg

from .lattice import exp_hopping


def slice_scales(x_col, dtau, lam):
    """Diagonal of exp(-dtau lam x_l)."""
    return np.exp(-dtau * lam * np.asarray(x_col, dtype=np.float64))


def slice_matrix(E, x_col, dtau, lam):
    """B_l = diag(exp(-dtau lam x_l)) E (Eq. (S2))."""
    return slice_scales(x_col, dtau, lam)[:, None] * E


def udt_chain(E, x, dtau, lam, n_s):
    """Stable factorisation B_L ... B_1 = U diag(D) T."""
    N, L = x.shape
    U = np.eye(N)
    D = np.ones(N)
    T = np.eye(N)
    for g0 in range(0, L, n_s):
        Y = U
        for l in range(g0, min(g0 + n_s, L)):
            Y = slice_matrix(E, x[:, l], dtau, lam) @ Y
        C = Y * D[None, :]
        Q, R, P = scipy.linalg.qr(C, pivoting=True)   # C[:, P] = Q R
        Dn = np.abs(np.diag(R))
        T = (R / Dn[:, None]) @ T[P, :]
        U, D = Q, Dn
    return U, D, T


def logdet_greens_from_udt(U, D, T):
    """ln|det(I + U D T)|, its sign and G = (I + U D T)^-1 through the D_b / D_s split."""
    Db = np.maximum(D, 1.0)
    Ds = np.minimum(D, 1.0)
    M = U.T / Db[:, None] + Ds[:, None] * T
    sM, lM = np.linalg.slogdet(M)
    sU, lU = np.linalg.slogdet(U)
    lndet = float(np.sum(np.log(Db)) + lM + lU)
    G = np.linalg.solve(M, U.T / Db[:, None])
    return lndet, int(np.sign(sM * sU)), G


def fermion_logdet(p, x, E=None, want_G=True):
    """(ln|det(I + B_L ... B_1)|, sign, G or None) for one field x[N, L]."""
    x = np.asarray(x, dtype=np.float64)
    assert x.shape == (p.N, p.L)
    if E is None:
        E = exp_hopping(p.Lx, p.Ly, p.t, p.mu, p.dtau)
    U, D, T = udt_chain(E, x, p.dtau, p.lam, p.n_s)
    lndet, sign, G = logdet_greens_from_udt(U, D, T)
    return lndet, sign, (G if want_G else None)


def block_matrix(E, x, dtau, lam):
    """The NL x NL matrix O with identity blocks on the diagonal, -B_l at block
    (l, l-1) for l = 2..L and +B_1 at block (1, L). det O = det(I + B_L ... B_1) and the
    (L, L) block of O^-1 is G(L) (used for brute-force pins on tiny lattices)."""
    N, L = x.shape
    O = np.eye(N * L)
    for l in range(1, L):
        O[l * N:(l + 1) * N, (l - 1) * N:l * N] = -slice_matrix(E, x[:, l], dtau, lam)
    O[0:N, (L - 1) * N:L * N] = slice_matrix(E, x[:, 0], dtau, lam)
    return O
