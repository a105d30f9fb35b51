"""Square lattice with periodic boundaries and the hopping matrix (oracle; test
infrastructure only).

Eq. (2), H_el: -t on every nearest-neighbour bond of the periodic Lx x Ly square
lattice, -mu on the diagonal. Site index i = ix + Lx * iy. Eq. (S2): the slice matrix
uses exp(-dtau K), computed here from the eigen-decomposition of the symmetric K
(a library eigensolver serves as the step).
"""
import numpy as np


def site(ix, iy, Lx):
    return ix + Lx * iy


def coords(N, Lx):
    i = np.arange(N)
    return i % Lx, i // Lx


def staggered_sign(Lx, Ly):
    """s_i = (-1)^(ix+iy), the (pi,pi) sublattice sign."""
    ix, iy = coords(Lx * Ly, Lx)
    return np.where((ix + iy) % 2 == 0, 1.0, -1.0)


def hopping_matrix(Lx, Ly, t, mu):
    """K of Eq. (2): K[i, j] = -t for each of the four periodic neighbour directions
    (on a length-2 side the +1 and -1 neighbours coincide and both bonds add), and
    K[i, i] = -mu."""
    N = Lx * Ly
    K = np.zeros((N, N))
    for iy in range(Ly):
        for ix in range(Lx):
            i = site(ix, iy, Lx)
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                j = site((ix + dx) % Lx, (iy + dy) % Ly, Lx)
                K[i, j] += -t
            K[i, i] += -mu
    return K


def exp_hopping(Lx, Ly, t, mu, dtau):
    """E = exp(-dtau K) via eigh (Eq. (S2))."""
    K = hopping_matrix(Lx, Ly, t, mu)
    w, V = np.linalg.eigh(K)
    return (V * np.exp(-dtau * w)[None, :]) @ V.T


def dispersion(Lx, Ly, t, mu):
    """Band energies eps_k = -2t (cos kx + cos ky) - mu for k = 2 pi (nx/Lx, ny/Ly),
    the eigenvalues of K (closed form used only as a test pin)."""
    kx = 2 * np.pi * np.arange(Lx) / Lx
    ky = 2 * np.pi * np.arange(Ly) / Ly
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    return (-2 * t * (np.cos(KX) + np.cos(KY)) - mu).ravel(), KX.ravel(), KY.ravel()
