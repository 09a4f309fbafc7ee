"""Seeded synthetic inputs for the Hartree step (atom positions, charges, cells).

This module only builds inputs: diamond lattice sites, seeded jitter, seeded
charges and seeded cell shapes.  It holds none of the method's arithmetic
(no splatting, no transforms, no Green function), so both the FP64 oracle and
the CUDA library can be fed from it without sharing any computation.

The benchmark systems of the paper are diamond crystals (Sec. 5.1.3); the
configurations below are diamond supercells of the conventional cubic cell,
lattice constant 6.74 Bohr (3.567 Angstrom), plus seeded perturbations.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` with
``seed = 1209_4506_0 * 10 + config_id`` unless a seed is given explicitly.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 120945060
DIAMOND_A = 6.74  # Bohr

# Fractional coordinates of the 8 sites of the conventional diamond cell:
# the four FCC sites and the same four shifted by (1/4, 1/4, 1/4).
DIAMOND_BASIS = np.array(
    [
        [0.00, 0.00, 0.00],
        [0.00, 0.50, 0.50],
        [0.50, 0.00, 0.50],
        [0.50, 0.50, 0.00],
        [0.25, 0.25, 0.25],
        [0.25, 0.75, 0.75],
        [0.75, 0.25, 0.75],
        [0.75, 0.75, 0.25],
    ],
    dtype=np.float64,
)


@dataclass
class System:
    """One periodic orthorhombic cell with Gaussian charges and its grid.

    Attributes:
      name: workload label.
      n: grid points (N1, N2, N3) along a, b, c; layout is C order, c fastest.
      cell: side lengths (L1, L2, L3) in Bohr.
      sigma: Gaussian width parameter in Bohr (density q (pi s^2)^-3/2 e^{-r^2/s^2}).
      pos: (n_atoms, 3) float64 positions in Bohr, wrapped into [0, L).
      q: (n_atoms,) float64 charges in e.
      precision: 'fp64', 'fp32' or 'bf16split'.
    """

    name: str
    n: Tuple[int, int, int]
    cell: Tuple[float, float, float]
    sigma: float
    pos: np.ndarray
    q: np.ndarray
    precision: str = "fp32"
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_tot(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def rng_for(config_id: int, seed: Optional[int] = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id if seed is None else seed))


def wrap(pos: np.ndarray, cell: Sequence[float]) -> np.ndarray:
    """Wrap positions into [0, L) per axis."""
    L = np.asarray(cell, dtype=np.float64)
    out = np.mod(pos, L)
    # np.mod can return L itself for tiny negative inputs; fold those to 0.
    return np.where(out >= L, out - L, out)


def diamond_supercell(reps: Tuple[int, int, int], a: float = DIAMOND_A) -> np.ndarray:
    """Sites of a reps[0] x reps[1] x reps[2] supercell of the conventional cell."""
    cells = np.stack(
        np.meshgrid(np.arange(reps[0]), np.arange(reps[1]), np.arange(reps[2]), indexing="ij"), axis=-1
    ).reshape(-1, 1, 3)
    return ((cells + DIAMOND_BASIS[None, :, :]) * a).reshape(-1, 3).astype(np.float64)


def diamond_in_box(cell: Sequence[float], a: float = DIAMOND_A) -> np.ndarray:
    """Diamond sites (lattice constant a) that fall inside [0, L1) x [0, L2) x [0, L3)."""
    L = np.asarray(cell, dtype=np.float64)
    reps = tuple(int(np.ceil(L[d] / a)) for d in range(3))
    sites = diamond_supercell(reps, a)
    keep = np.all(sites < L[None, :], axis=1)
    return sites[keep]


def jitter(rng: np.random.Generator, pos: np.ndarray, amount: float, cell) -> np.ndarray:
    """Each Cartesian component moved by U(-amount, +amount), then wrapped."""
    return wrap(pos + rng.uniform(-amount, amount, size=pos.shape), cell)


def centred_uniform_charges(rng: np.random.Generator, n: int) -> np.ndarray:
    """q ~ U(-1, 1), then shifted by its mean so the cell is neutral."""
    q = rng.uniform(-1.0, 1.0, size=n)
    return q - q.mean() if n > 0 else q


def smooth235(x: float, even: bool = True) -> int:
    """Smallest integer >= x whose only prime factors are 2, 3, 5 (even if asked)."""
    m = max(1, int(np.ceil(x - 1e-9)))
    while True:
        v = m
        for p in (2, 3, 5):
            while v % p == 0:
                v //= p
        if v == 1 and (not even or m % 2 == 0):
            return m
        m += 1


# ---------------------------------------------------------------- configurations
def config1(seed: Optional[int] = None) -> System:
    """8-atom conventional diamond cell, a = 6.74 Bohr, 32^3 grid, FP64, q = +1/-1 alternating."""
    rng = rng_for(1, seed)
    cell = (DIAMOND_A,) * 3
    pos = jitter(rng, diamond_supercell((1, 1, 1)), 0.05, cell)
    q = np.array([1.0 if i % 2 == 0 else -1.0 for i in range(8)])
    return System("diamond-1x1x1 32^3 fp64", (32, 32, 32), cell, 0.8, pos, q, "fp64")


def config2(seed: Optional[int] = None) -> System:
    """64-atom 2x2x2 diamond supercell, a = 13.48 Bohr, 120^3 grid, FP32."""
    rng = rng_for(2, seed)
    cell = (2 * DIAMOND_A,) * 3
    pos = jitter(rng, diamond_supercell((2, 2, 2)), 0.1, cell)
    q = centred_uniform_charges(rng, pos.shape[0])
    return System("diamond-2x2x2 120^3 fp32", (120, 120, 120), cell, 0.6, pos, q, "fp32")


def config3a(seed: Optional[int] = None) -> System:
    """4096-atom 8x8x8 diamond supercell, a = 53.92 Bohr, 512^3 grid, FP32 (headline)."""
    rng = rng_for(3, seed)
    cell = (8 * DIAMOND_A,) * 3
    pos = jitter(rng, diamond_supercell((8, 8, 8)), 0.1, cell)
    q = centred_uniform_charges(rng, pos.shape[0])
    return System("diamond-8x8x8 512^3 fp32", (512, 512, 512), cell, 0.5, pos, q, "fp32")


def config3b(seed: Optional[int] = None) -> System:
    """Orthorhombic 37.9 x 40.4 x 42.1 Bohr cell, 360 x 384 x 400 grid, diamond density, FP32."""
    rng = rng_for(33, seed)
    cell = (37.9, 40.4, 42.1)
    pos = jitter(rng, diamond_in_box(cell), 0.1, cell)
    q = centred_uniform_charges(rng, pos.shape[0])
    return System("diamond-ortho 360x384x400 fp32", (360, 384, 400), cell, 0.5, pos, q, "fp32")


def config_paper420(seed: Optional[int] = None) -> System:
    """16x16x8 diamond supercell (16,384 atoms, 107.84 x 107.84 x 53.92 Bohr) on 420 x 420 x 210.

    This is the grid of the paper's memory benchmark of the 16,384-atom diamond system (Sec. 5.2.6),
    at its spacing of about 0.257 Bohr (the 150 Ry cutoff of Sec. 5.1.1).  Radix 7 on every axis.
    sigma = 0.8 Bohr keeps the Gaussians resolved at that spacing.  FP32."""
    rng = rng_for(6, seed)
    cell = (16 * DIAMOND_A, 16 * DIAMOND_A, 8 * DIAMOND_A)
    pos = jitter(rng, diamond_supercell((16, 16, 8)), 0.1, cell)
    q = centred_uniform_charges(rng, pos.shape[0])
    return System("diamond-16x16x8 420x420x210 fp32", (420, 420, 210), cell, 0.8, pos, q, "fp32")


def config_paper420cube(seed: Optional[int] = None) -> System:
    """16x16x16 diamond supercell (32,768 atoms, a 107.84 Bohr cube) on 420^3: the paper's
    32,768-atom memory benchmark grid (Sec. 5.2.6) at its spacing of about 0.257 Bohr.  sigma = 0.8
    Bohr as on the 420 x 420 x 210 grid.  FP32."""
    rng = rng_for(7, seed)
    cell = (16 * DIAMOND_A,) * 3
    pos = jitter(rng, diamond_supercell((16, 16, 16)), 0.1, cell)
    q = centred_uniform_charges(rng, pos.shape[0])
    return System("diamond-16x16x16 420^3 fp32", (420, 420, 420), cell, 0.8, pos, q, "fp32")


def config_paper840(seed: Optional[int] = None) -> System:
    """32x16x16 diamond supercell (65,536 atoms, 215.68 x 107.84 x 107.84 Bohr) on 840 x 420 x 420: the
    paper's 65,536-atom memory benchmark grid (Sec. 5.2.6) at about 0.257 Bohr.  sigma = 0.8 Bohr.
    FP32."""
    rng = rng_for(8, seed)
    cell = (32 * DIAMOND_A, 16 * DIAMOND_A, 16 * DIAMOND_A)
    pos = jitter(rng, diamond_supercell((32, 16, 16)), 0.1, cell)
    q = centred_uniform_charges(rng, pos.shape[0])
    return System("diamond-32x16x16 840x420x420 fp32", (840, 420, 420), cell, 0.8, pos, q, "fp32")


def config4(seed: Optional[int] = None, n_cells: int = 64) -> List[System]:
    """64 independent orthorhombic cells, edges U(8, 30) Bohr, 0.17 Bohr spacing, 8..1000 atoms."""
    rng = rng_for(4, seed)
    out = []
    for c in range(n_cells):
        cell = tuple(float(x) for x in rng.uniform(8.0, 30.0, size=3))
        n = tuple(int(min(180, max(48, smooth235(L / 0.17)))) for L in cell)
        nat = int(rng.integers(8, 1001))
        pos = wrap(rng.uniform(0.0, 1.0, size=(nat, 3)) * np.asarray(cell)[None, :], cell)
        q = centred_uniform_charges(rng, nat)
        out.append(System(f"batch-cell-{c}", n, cell, 0.6, pos, q, "fp32"))
    return out


def config5(seed: Optional[int] = None) -> System:
    """512-atom 4x4x4 diamond supercell, a = 26.96 Bohr, 256^3 grid, BF16-split radix-16 stage."""
    rng = rng_for(5, seed)
    cell = (4 * DIAMOND_A,) * 3
    pos = jitter(rng, diamond_supercell((4, 4, 4)), 0.1, cell)
    q = centred_uniform_charges(rng, pos.shape[0])
    return System("diamond-4x4x4 256^3 bf16split", (256, 256, 256), cell, 0.5, pos, q, "bf16split")


def random_system(
    n: Tuple[int, int, int],
    cell: Tuple[float, float, float],
    n_atoms: int,
    sigma: float,
    seed: int,
    precision: str = "fp64",
    neutral: bool = True,
) -> System:
    """Uniformly placed Gaussian charges in an arbitrary orthorhombic cell (test cases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = wrap(rng.uniform(0.0, 1.0, size=(n_atoms, 3)) * np.asarray(cell)[None, :], cell)
    q = centred_uniform_charges(rng, n_atoms) if neutral else rng.uniform(-1.0, 1.0, size=n_atoms)
    return System(f"random-{n}-{n_atoms}", tuple(n), tuple(cell), sigma, pos, q, precision)


CONFIGS = {
    "cfg1": config1,
    "cfg2": config2,
    "cfg3a": config3a,
    "cfg3b": config3b,
    "cfg5": config5,
    "paper420": config_paper420,
}
