"""Seeded synthetic phonon fields shared by the tests, the oracle comparisons and the
benchmark. Holds no arithmetic of the method: only random draws and the site layout
i = ix + Lx * iy of x[n][N][L] (row-major, float64).

The paper's DQMC configurations are not available, so these synthetic fields stand in:
iid Gaussian fields, and a checkerboard CDW pattern amp * (-1)^(ix+iy) (constant in
imaginary time) plus Gaussian noise, the ordered shape the Holstein model develops below
its CDW transition.
"""
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.Philox(int(seed) & ((1 << 64) - 1)))


def gaussian_fields(n, Lx, Ly, L, sigma=1.0, seed=0):
    return sigma * _rng(seed).standard_normal((n, Lx * Ly, L))


def cdw_fields(n, Lx, Ly, L, amp=0.8, noise=0.3, seed=0):
    i = np.arange(Lx * Ly)
    stag = np.where(((i % Lx) + (i // Lx)) % 2 == 0, 1.0, -1.0)
    return amp * stag[None, :, None] + noise * _rng(seed).standard_normal((n, Lx * Ly, L))


def mixed_fields(n, Lx, Ly, L, seed=0):
    """First half iid N(0, 1), second half CDW 0.8 (-1)^(ix+iy) + N(0, 0.3^2)."""
    h = n // 2
    return np.concatenate([gaussian_fields(h, Lx, Ly, L, 1.0, seed),
                           cdw_fields(n - h, Lx, Ly, L, 0.8, 0.3, seed + 1)], axis=0)
