"""Seeded synthetic inputs for the FeGe B20 workloads.

This module only builds input arrays (positions, spins, species, velocities,
boxes, field/temperature schedules).  It holds none of the potential's or the
integrator's arithmetic, so both the CUDA path and the CPU oracle draw their
inputs from here.

Structure (an assumption, the paper fixes only the material and its helix):
B20 FeGe, space group P2_13, cubic a = 4.70 A, 4 Fe + 4 Ge per cell on the 4a
Wyckoff sites (u,u,u), (1/2+u, 1/2-u, -u), (-u, 1/2+u, 1/2-u), (1/2-u, -u, 1/2+u)
with u_Fe = 0.135 and u_Ge = 0.842.  The paper's benchmark (Section 6.2) drives
a helical FeGe state; one unit spin per atom (Section 3).

Atom order returned to callers: cell-major (x fastest), inside a cell the four
Fe sites then the four Ge sites.  Species codes: Fe = 0, Ge = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

A_FEGE = 4.70                  # cubic lattice constant, Angstrom
U_FE = 0.135
U_GE = 0.842
MASS_AMU = (55.845, 72.630)    # Fe, Ge
MOMENT_MUB = (1.0, 1.0)        # one Bohr magneton per atom (reading; paper gives none)
KB_EV = 8.617333262e-5         # Boltzmann constant, eV/K (CODATA 2018)
EV_PER_AMU_A2_FS2 = 1.0 / 9.6485332e-3   # (amu A^2/fs^2) -> eV

STRUCTURE_SEED0 = 20260101      # + workload id
PARAM_SEED = 7
LANGEVIN_SEED0 = 1234           # + replica id


def _b20_sites(u: float) -> np.ndarray:
    return np.array([[u, u, u],
                     [0.5 + u, 0.5 - u, -u],
                     [-u, 0.5 + u, 0.5 - u],
                     [0.5 - u, -u, 0.5 + u]], dtype=np.float64) % 1.0


def b20_lattice(nx: int, ny: int, nz: int, a: float = A_FEGE):
    """Perfect B20 FeGe crystal of nx*ny*nz cells.

    Returns (positions [N,3] A, species [N] int32, box [3] A).
    """
    frac = np.concatenate([_b20_sites(U_FE), _b20_sites(U_GE)])       # [8,3]
    spec = np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.int32)
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.float64)   # x fastest
    pos = (cells[:, None, :] + frac[None, :, :]).reshape(-1, 3) * a
    species = np.tile(spec, cells.shape[0])
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return pos, species, box


def wrap(pos: np.ndarray, box: np.ndarray, periodic) -> np.ndarray:
    out = pos.copy()
    for d in range(3):
        if periodic[d]:
            out[:, d] = out[:, d] - box[d] * np.floor(out[:, d] / box[d])
    return out


def random_unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def maxwell_boltzmann(rng: np.random.Generator, species: np.ndarray, T: float) -> np.ndarray:
    """Velocities in A/fs at temperature T (K), net momentum removed."""
    m = np.asarray(MASS_AMU, dtype=np.float64)[species]
    if T <= 0.0:
        return np.zeros((species.shape[0], 3))
    sigma = np.sqrt(KB_EV * T / (m * EV_PER_AMU_A2_FS2))
    v = rng.standard_normal((species.shape[0], 3)) * sigma[:, None]
    p = (m[:, None] * v).sum(axis=0)
    v -= p[None, :] / m.sum()
    return v


@dataclasses.dataclass
class Workload:
    name: str
    positions: np.ndarray      # [N,3] float64, A
    spins: np.ndarray          # [N,3] float64, unit vectors
    species: np.ndarray        # [N] int32
    velocities: np.ndarray     # [N,3] float64, A/fs
    box: np.ndarray            # [3] float64, A
    periodic: np.ndarray       # [3] int32
    T: float                   # K
    B: np.ndarray              # [3] tesla
    dt: float                  # fs
    n_steps: int
    seed: int                  # Langevin / spin-noise key

    @property
    def n(self) -> int:
        return int(self.positions.shape[0])


def fege_cube(cells: int, *, T: float = 300.0, jitter: float = 0.02, spin_mode: str = "random",
              cant_deg: float = 5.0, seed: int = STRUCTURE_SEED0 + 1, B=(0.0, 0.0, 0.0),
              dt: float = 1.0, n_steps: int = 100, name: str | None = None,
              replica: int = 0) -> Workload:
    """Periodic cube of cells^3 B20 cells.

    spin_mode "random": spins uniform on the sphere; "canted": z tilted by cant_deg
    towards a uniform random azimuth per atom.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pos, species, box = b20_lattice(cells, cells, cells)
    pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    periodic = np.array([1, 1, 1], dtype=np.int32)
    pos = wrap(pos, box, periodic)
    n = pos.shape[0]
    if spin_mode == "random":
        spins = random_unit_vectors(rng, n)
    elif spin_mode == "canted":
        phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
        th = math.radians(cant_deg)
        spins = np.stack([math.sin(th) * np.cos(phi), math.sin(th) * np.sin(phi),
                          np.full(n, math.cos(th))], axis=1)
    else:
        raise ValueError(spin_mode)
    vel = maxwell_boltzmann(rng, species, T)
    return Workload(name or f"fege_b20_{cells}c", pos, spins, species, vel, box, periodic, T,
                    np.asarray(B, dtype=np.float64), dt, n_steps, LANGEVIN_SEED0 + replica)


def fege_small(seed_offset: int = 1) -> Workload:
    """4x4x4 cells = 512 atoms, jittered, random spins, 300 K, 100 steps of 1 fs."""
    return fege_cube(4, T=300.0, spin_mode="random", seed=STRUCTURE_SEED0 + seed_offset,
                     n_steps=100, name="fege_b20_4c_512")


def fege_884k() -> Workload:
    """48x48x48 cells = 884,736 atoms, ferromagnetic z with a 5 degree random cant, 300 K."""
    return fege_cube(48, T=300.0, spin_mode="canted", seed=STRUCTURE_SEED0 + 2,
                     n_steps=1000, name="fege_b20_48c_884736")


def fege_slab_helix(nx: int = 160, ny: int = 160, nz: int = 16, *, vacuum: float = 10.0,
                    period_target: float = 700.0, B_z: float = 0.2, seed: int = STRUCTURE_SEED0 + 3,
                    T: float = 0.0) -> Workload:
    """Slab periodic in x,y with free z surfaces and a helix along x.

    The helix period is the box length divided by the whole number of turns
    closest to period_target (A), so the texture is continuous across x.
    The binning extent in z is the slab thickness plus vacuum on both sides.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pos, species, box = b20_lattice(nx, ny, nz)
    pos = pos + rng.normal(0.0, 0.02, size=pos.shape)
    pos[:, 2] += vacuum
    box = box.copy()
    box[2] = box[2] + 2.0 * vacuum
    periodic = np.array([1, 1, 0], dtype=np.int32)
    pos = wrap(pos, box, periodic)
    turns = max(1, int(round(box[0] / period_target)))
    lam = box[0] / turns
    ph = 2.0 * math.pi * pos[:, 0] / lam
    spins = np.stack([np.zeros_like(ph), np.cos(ph), np.sin(ph)], axis=1)
    vel = maxwell_boltzmann(rng, species, T)
    return Workload(f"fege_slab_{nx}x{ny}x{nz}_helix", pos, spins, species, vel, box, periodic, T,
                    np.array([0.0, 0.0, B_z]), 1.0, 20000, LANGEVIN_SEED0)


def isolated_cluster(n_side: int = 2, seed: int = 99, jitter: float = 0.15):
    """Small non-periodic B20 fragment with random spins (for invariance pins)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos, species, box = b20_lattice(n_side, n_side, n_side)
    pos = pos + rng.normal(0.0, jitter, size=pos.shape) + 20.0
    spins = random_unit_vectors(rng, pos.shape[0])
    box = np.array([100.0, 100.0, 100.0])
    return pos, spins, species, box, np.array([0, 0, 0], dtype=np.int32)


def replica_sizes(count: int = 64, seed: int = STRUCTURE_SEED0 + 4):
    """Uneven replica family: atoms log-uniform in [4096, 262144], cells per side
    = clamp(round((N/8)^(1/3)), 8, 32); T ~ U(100,300) K; B_z ~ U(0,0.5) T."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = np.exp(rng.uniform(math.log(4096), math.log(262144), size=count))
    cells = np.clip(np.rint(np.cbrt(n / 8.0)), 8, 32).astype(int)
    T = rng.uniform(100.0, 300.0, size=count)
    Bz = rng.uniform(0.0, 0.5, size=count)
    return cells, T, Bz
