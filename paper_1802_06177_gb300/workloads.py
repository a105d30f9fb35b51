"""The benchmark workloads, named by what they are (model parameters t = 1, mu = 0,
omega0 = 1, lambda = 1, dtau = 0.1 throughout; beta = L * dtau)."""
from dataclasses import dataclass


@dataclass(frozen=True)
class Workload:
    name: str
    Lx: int
    L: int
    n_s: int
    nfields: int
    fields: str          # "gaussian" or "mixed" (half Gaussian, half CDW + noise)
    nsweeps: int = 50
    nupdates: int = 0
    seed: int = 0x1802061770

    @property
    def N(self):
        return self.Lx * self.Lx

    @property
    def beta(self):
        return self.L * 0.1


WORKLOADS = {
    "holstein_4x4_L40": Workload("holstein_4x4_L40", 4, 40, 10, 64, "gaussian", 50, 200, 0x1802061770),
    "holstein_12x12_L120": Workload("holstein_12x12_L120", 12, 120, 10, 256, "mixed", seed=0x1802061771),
    "holstein_16x16_L160": Workload("holstein_16x16_L160", 16, 160, 8, 512, "mixed", seed=0x1802061772),
    "holstein_24x24_L240": Workload("holstein_24x24_L240", 24, 240, 8, 32, "gaussian", 100, 500, 0x1802061774),
}

# Uneven batch of independent chains: (Lx, L, count).
UNEVEN_BATCH = ((8, 80, 64), (10, 100, 64), (12, 120, 64), (16, 160, 64))
