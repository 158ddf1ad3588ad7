"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the homogenisation method itself: it only
draws random numbers and lays out inputs (a periodic Voronoi grain map, grain
orientations as unit quaternions, material constants, a macroscopic load
programme).  Both the FP64 CPU oracle and the CUDA path consume the arrays it
returns; neither side's arithmetic lives here.

The paper (Sec. 2.2) builds its RVEs with Dream3D (equiaxed grains, lognormal
sizes, random texture); the synthetic stand-in used here is a periodic
Voronoi tessellation of seeded uniform points in the unit cube with uniformly
random orientations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014; constants as published by Vigna)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1): the top 53 bits times 2^-53."""
        return np.array([(self.next_u64() >> 11) * (2.0 ** -53) for _ in range(n)],
                        dtype=np.float64)


def voronoi_grain_map(n: int, n_grains: int, seed: int, shape=None) -> tuple[np.ndarray, np.ndarray]:
    """Periodic Voronoi grain map on an n0 x n1 x n2 voxel grid.

    Returns (grain_id, seeds).  grain_id has numpy shape (n2, n1, n0), i.e. x is the
    fastest index (linear voxel index = x + n0*(y + n1*z)), dtype int32.  Voxel
    centres sit at ((i+1/2)/n0, ...) in the unit periodic cube; each voxel goes
    to the seed at the smallest minimum-image Euclidean distance, ties to the
    lowest grain id.
    """
    rng = SplitMix64(seed)
    seeds = rng.uniform(3 * n_grains).reshape(n_grains, 3)
    n0, n1, n2 = shape if shape is not None else (n, n, n)
    xs = (np.arange(n0) + 0.5) / n0
    ys = (np.arange(n1) + 0.5) / n1
    zs = (np.arange(n2) + 0.5) / n2
    best = np.full((n2, n1, n0), np.inf)
    gid = np.zeros((n2, n1, n0), dtype=np.int32)
    for g in range(n_grains):
        dx = np.abs(xs - seeds[g, 0]); dx = np.minimum(dx, 1.0 - dx)
        dy = np.abs(ys - seeds[g, 1]); dy = np.minimum(dy, 1.0 - dy)
        dz = np.abs(zs - seeds[g, 2]); dz = np.minimum(dz, 1.0 - dz)
        d2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        better = d2 < best          # strict: an equal distance keeps the lower id
        best[better] = d2[better]
        gid[better] = g
    return gid, seeds


def random_quaternions(n_grains: int, seed: int) -> np.ndarray:
    """Uniformly random unit quaternions (w, x, y, z), Shoemake's method
    (Graphics Gems III, 1992): three uniforms u1, u2, u3."""
    rng = SplitMix64(seed)
    u = rng.uniform(3 * n_grains).reshape(n_grains, 3)
    u1, u2, u3 = u[:, 0], u[:, 1], u[:, 2]
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    qx = a * np.sin(2 * math.pi * u2)
    qy = a * np.cos(2 * math.pi * u2)
    qz = b * np.sin(2 * math.pi * u3)
    qw = b * np.cos(2 * math.pi * u3)
    return np.stack([qw, qx, qy, qz], axis=1)


# ---------------------------------------------------------------------------
# Material constants.  Elastic constants and Burgers vectors are the values the
# workloads prescribe; the similitude coefficient K and the annihilation
# distance y_c are the paper's Table 2; the viscoplastic parameters and the
# six interaction coefficients are Table 1 (exponent n = 1/m = 20).
# Units: MPa for moduli and stresses, metres for lengths, m^-2 for densities.
# ---------------------------------------------------------------------------
Q_TABLE1 = (0.122, 0.122, 0.657, 0.084, 0.137, 0.118)  # self, coplanar, collinear, Hirth, glissile, Lomer


@dataclass
class Material:
    C11: float
    C12: float
    C44: float
    b: float
    tau0: float
    K: float
    yc: float
    alpha: float = 0.3
    q: tuple = Q_TABLE1
    q_normalise: bool = True      # q_hat = q / q_self, so the self term is 1
    gdot0: float = 1.0e-3
    n: float = 20.0
    rho0_total: float = 1.0e12
    mu: float = 0.0               # 0: derive from the cubic constants
    gnd_enabled: bool = True

    def asdict(self):
        return asdict(self)


PRESETS = {
    "Cu": dict(C11=168.4e3, C12=121.4e3, C44=75.4e3, b=0.256e-9, tau0=10.0, K=6.0, yc=15e-9),
    "Al": dict(C11=108.2e3, C12=61.3e3, C44=28.5e3, b=0.286e-9, tau0=5.0, K=9.0, yc=56e-9),
    "Ag": dict(C11=124.0e3, C12=93.4e3, C44=46.1e3, b=0.289e-9, tau0=10.0, K=5.0, yc=12.5e-9),
    "Ni": dict(C11=246.5e3, C12=147.3e3, C44=124.7e3, b=0.249e-9, tau0=10.0, K=11.0, yc=14e-9),
}


def material(name: str, **over) -> Material:
    d = dict(PRESETS[name]); d.update(over)
    return Material(**d)


# ---------------------------------------------------------------------------
# Workloads.  Uniaxial tension along x: F11 prescribed (engineering strain
# rate), F21, F31, F32 held at 0 (fixes the rigid rotation), P22, P33, P12,
# P13, P23 held at 0.  Row-major 3x3 index 3*i + j.
# ---------------------------------------------------------------------------
UNIAXIAL_X_MASK = np.array([1, 0, 0, 1, 0, 0, 1, 1, 0], dtype=np.uint8)  # 1 = strain-controlled


@dataclass
class Workload:
    name: str
    n: int
    n_grains: int
    material: str
    strain: float
    increments: int
    rate: float = 1.0e-3
    seed: int = 1000
    mean_grain_um: float = 20.0      # sphere-equivalent mean grain diameter
    L: float = 0.0                   # RVE edge [m]; 0 = from mean_grain_um

    @property
    def dt(self) -> float:
        return self.strain / (self.rate * self.increments)

    @property
    def edge(self) -> float:
        if self.L > 0:
            return self.L
        return self.mean_grain_um * 1e-6 * (math.pi * self.n_grains / 6.0) ** (1.0 / 3.0)

    def dFbar(self) -> np.ndarray:
        d = np.zeros(9); d[0] = self.rate * self.dt
        return d

    def inputs(self):
        gid, _ = voronoi_grain_map(self.n, self.n_grains, self.seed)
        quat = random_quaternions(self.n_grains, self.seed + 7919)
        return gid, quat, material(self.material)


WORKLOADS = {
    "cu16": Workload("cu16_8g_1pct_20inc", 16, 8, "Cu", 0.01, 20, seed=1000),
    "cu64": Workload("cu64_100g_5pct_50inc", 64, 100, "Cu", 0.05, 50, seed=1001),
    "al128": Workload("al128_500g_3pct_30inc", 128, 500, "Al", 0.03, 30, seed=1002),
    # the calibration workload: stress curve and its sensitivities to (tau0, K, alpha, b)
    "cu64g64": Workload("cu64_64g_2pct_20inc", 64, 64, "Cu", 0.02, 20, seed=1004),
}


def sweep_workloads():
    """The batched grain-size sweep: 16 RVEs j = 0..15 with edge
    {32, 48, 64, 96}[j // 4] voxels, n_j = round(8 * 50^(j/15)) grains (8 to
    400, log-spaced), materials Cu, Al, Ag, Ni cycled, a fixed 100 um edge (so
    the mean grain size falls from about 62 to 17 um), tension to 2 % in 20
    increments at 1e-3 /s, seeds 1300 + j."""
    out = []
    for j in range(16):
        n = (32, 48, 64, 96)[j // 4]
        g = int(round(8 * 50 ** (j / 15.0)))
        out.append(Workload(f"sweep{j:02d}_{n}_{g}g_{('Cu', 'Al', 'Ag', 'Ni')[j % 4]}", n, g,
                            ("Cu", "Al", "Ag", "Ni")[j % 4], 0.02, 20, seed=1300 + j, L=100e-6))
    return out


def bicrystal_slip_jump(n: int, gamma: float = 1e-3) -> np.ndarray:
    """A plastic distortion that jumps across grain boundaries (the input of
    the Gibbs comparison of the Nye tensor): two slabs along x, x < n/2 with
    the single slip Fp = I + gamma s (x) m on the system s = [-1 0 1]/sqrt 2,
    m = (1 1 1)/sqrt 3, and x >= n/2 with Fp = I.  Numpy shape
    (n, n, n, 3, 3) = (z, y, x, i, j)."""
    s = np.array([-1.0, 0.0, 1.0]) / math.sqrt(2.0)
    m = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    Fp = np.tile(np.eye(3), (n, n, n, 1, 1)).astype(np.float64)
    Fp[:, :, : n // 2] += gamma * np.outer(s, m)
    return Fp
