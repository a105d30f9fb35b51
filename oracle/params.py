"""Model and discretisation parameters (oracle copy; test infrastructure only).

Eq. (1)-(2): Holstein model with hopping t, chemical potential mu, phonon frequency
omega0 (the paper's Omega, with M = 1) and coupling lam (the paper's g). The coupling is
taken in the particle-hole symmetric form lam * x_i * (n_i - 1), i.e. the paper's field
shifted by its mirror axis alpha = -g/Omega^2 (Sec. "Designing the effective model"), so
the two phonon minima of the atomic limit sit at x = +-a with a = lam / omega0^2.
Eq. (S1): beta = L * dtau with L imaginary-time slices.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class HolsteinParams:
    Lx: int
    Ly: int
    L: int            # number of imaginary-time slices
    dtau: float = 0.1
    t: float = 1.0
    mu: float = 0.0
    omega0: float = 1.0
    lam: float = 1.0
    n_s: int = 10     # slices multiplied between two stabilisations

    @property
    def N(self) -> int:
        return self.Lx * self.Ly

    @property
    def beta(self) -> float:
        return self.L * self.dtau

    @property
    def a(self) -> float:
        """Distance of each double-well minimum from the mirror axis, |alpha| = g/Omega^2."""
        return self.lam / self.omega0 ** 2
