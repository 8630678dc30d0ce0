"""Seeded synthetic inputs for the Poisson-Fermi solver.

This module only draws random numbers and lays out geometry (dielectric map, solvent
mask, charge positions, species tables, right-hand sides).  It holds none of the PF
method's arithmetic: unit conversions, charge spreading, operators and solvers live in
the CUDA library and, independently, in the CPU oracle.  Both sides take their inputs
from here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, 2014) used as a counter-based
generator: the k-th draw of a stream with seed s is mix(s + (k+1) * 0x9E3779B97F4A7C15),
uniforms take the top 53 bits, normals use the Box-Muller transform.

The paper's NCX workload (PDB 3v5u with PDB2PQR charges) is not available; the channel
problems below stand in for it with the same structure: a low-dielectric membrane slab,
water-filled pores, fixed charges on the pore walls and Dirichlet potentials on the two
bath planes (Eq. 4 of the paper).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of the SplitMix64 stream with the given seed (uint64)."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def substream(seed: int, tag: int) -> int:
    """A seed for an independent stream derived from (seed, tag)."""
    return int(splitmix64(seed ^ (tag * 0x632BE59BD9B4E019 & 0xFFFFFFFFFFFFFFFF), 1)[0])


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, n: int) -> np.ndarray:
    u = uniform(seed, 2 * n)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def to_f32_exact(a: np.ndarray) -> np.ndarray:
    """Round to the nearest float32 and return as float64, so float32 storage is lossless."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    h: float
    origin: tuple  # (x0, y0, z0) in Angstrom: coordinate of node (0,0,0)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape_zyx(self):
        return (self.nz, self.ny, self.nx)

    def coords(self):
        """Node coordinates as three (nz, ny, nx) arrays (x fastest in memory)."""
        x = self.origin[0] + self.h * np.arange(self.nx)
        y = self.origin[1] + self.h * np.arange(self.ny)
        z = self.origin[2] + self.h * np.arange(self.nz)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X, Y, Z


@dataclass
class Species:
    z: int
    radius_A: float
    bulk_M: float
    name: str = ""


NA = Species(+1, 0.95, 0.1, "Na+")
CL = Species(-1, 1.81, 0.1, "Cl-")
WATER = Species(0, 1.4, 55.5, "H2O")


@dataclass
class PFProblem:
    """One nonlinear PF problem: geometry, fixed charges, bath and boundary data."""
    grid: Grid
    eps: np.ndarray            # (N,) float64 relative dielectric at nodes
    solvent: np.ndarray        # (N,) uint8, 1 = solvent node
    charges: np.ndarray        # (M, 4) float64: x, y, z (A), q (e)
    phi_lo_V: float            # Dirichlet potential on the plane k = 0
    phi_hi_V: float            # Dirichlet potential on the plane k = nz-1
    species: list = field(default_factory=list)  # water last
    eps_s: float = 78.5
    lc_A: float = 1.2
    T_K: float = 298.15
    name: str = ""


@dataclass
class LinearProblem:
    """A variable-dielectric linear system (operator of Eq. 13 with no reaction term)."""
    grid: Grid
    eps: np.ndarray
    b: np.ndarray
    name: str = ""


def _channel_geometry(grid: Grid, slab_half: float, pores, eps_m: float, eps_s: float):
    X, Y, Z = grid.coords()
    in_pore = np.zeros(grid.shape_zyx, dtype=bool)
    for (cx, cy, r) in pores:
        in_pore |= (X - cx) ** 2 + (Y - cy) ** 2 < r * r
    membrane = (np.abs(Z) < slab_half) & ~in_pore
    solvent = (~membrane).astype(np.uint8).ravel()
    eps = np.where(membrane, eps_m, eps_s).astype(np.float64).ravel()
    return to_f32_exact(eps), solvent


def _wall_charges(seed: int, pores, count: int, slab_half: float, q_abs: float = 0.5):
    th = uniform(substream(seed, 1), count, 0.0, 2.0 * math.pi)
    zz = uniform(substream(seed, 2), count, -slab_half, slab_half)
    out = np.zeros((count, 4))
    for j in range(count):
        cx, cy, r = pores[j % len(pores)]
        out[j, 0] = cx + r * math.cos(th[j])
        out[j, 1] = cy + r * math.sin(th[j])
        out[j, 2] = zz[j]
        out[j, 3] = q_abs if j < count // 2 else -q_abs
    return out


def channel_problem(n: int = 33, box_half: float = 16.0, slab_half: float = 8.0, pores=((0.0, 0.0, 5.0),),
                    n_charges: int = 8, charge_seed: int = 0, phi_hi_V: float = 0.05, phi_lo_V: float = 0.0,
                    species=None, eps_m: float = 2.0, eps_s: float = 78.5, lc_A: float = 1.2,
                    name: str = "channel") -> PFProblem:
    """Membrane slab |z| < slab_half (eps_m) with cylindrical pores, bath eps_s, n^3 nodes on
    [-box_half, box_half]^3, charges of +-0.5 e on the pore walls (first half positive)."""
    h = 2.0 * box_half / (n - 1)
    grid = Grid(n, n, n, h, (-box_half, -box_half, -box_half))
    eps, solvent = _channel_geometry(grid, slab_half, pores, eps_m, eps_s)
    charges = _wall_charges(charge_seed, list(pores), n_charges, slab_half)
    sp = list(species) if species is not None else [NA, CL, WATER]
    return PFProblem(grid, eps, solvent, charges, phi_lo_V, phi_hi_V, sp, eps_s, lc_A, 298.15, name)


def config0() -> PFProblem:
    """33^3, h = 1 A, one pore of radius 5 A, 8 wall charges (seed 0), 0.1 M NaCl, 50 mV."""
    return channel_problem(33, name="pf_33_single_pore")


def config2(n: int = 257, seed: int = 2) -> PFProblem:
    """257^3 on [-32, 32]^3 A (h = 0.25 A), membrane slab |z| < 8 A with 4 pores centred at
    (+-10, +-10) A of radius U[4, 6] A, 48 wall charges, 0.1 M NaCl + 1 mM CaCl2, 50 mV."""
    radii = uniform(substream(seed, 7), 4, 4.0, 6.0)
    centres = [(10.0, 10.0), (-10.0, 10.0), (-10.0, -10.0), (10.0, -10.0)]
    pores = tuple((cx, cy, float(r)) for (cx, cy), r in zip(centres, radii))
    sp = [Species(+1, 0.95, 0.1, "Na+"), Species(+2, 0.99, 0.001, "Ca2+"),
          Species(-1, 1.81, 0.102, "Cl-"), WATER]
    return channel_problem(n, box_half=32.0, slab_half=8.0, pores=pores, n_charges=48,
                           charge_seed=substream(seed, 8), species=sp,
                           name=f"pf_{n}_four_pores_NaCaCl")


def linear_problem(n: int = 129, seed: int = 1, n_spheres: int = 32, h: float = 1.0) -> LinearProblem:
    """Variable-dielectric Poisson system: eps = 40 exp(0.5 g), g ~ N(0,1) iid per node, then
    n_spheres spheres (centres uniform in the box, radius U[4, 12] A) overwrite eps with 2 and
    78.5 alternately; right-hand side U[-1, 1] off the two Dirichlet planes, 0 on them."""
    half = 0.5 * h * (n - 1)
    grid = Grid(n, n, n, h, (-half, -half, -half))
    eps = 40.0 * np.exp(0.5 * normal(substream(seed, 1), grid.n))
    eps = eps.reshape(grid.shape_zyx)
    X, Y, Z = grid.coords()
    cen = uniform(substream(seed, 2), 3 * n_spheres, -half, half).reshape(n_spheres, 3)
    rad = uniform(substream(seed, 3), n_spheres, 4.0, 12.0)
    for s in range(n_spheres):
        inside = (X - cen[s, 0]) ** 2 + (Y - cen[s, 1]) ** 2 + (Z - cen[s, 2]) ** 2 < rad[s] ** 2
        eps[inside] = 2.0 if s % 2 == 0 else 78.5
    b = uniform(substream(seed, 4), grid.n, -1.0, 1.0).reshape(grid.shape_zyx)
    b[0] = 0.0
    b[-1] = 0.0
    return LinearProblem(grid, to_f32_exact(eps.ravel()), b.ravel().copy(), name=f"poisson_{n}_lognormal_spheres")


def batch_instances(count: int = 64, seed: int = 3, sizes=(33, 49, 65, 97)):
    """Independent channel problems on [-16, 16]^3 with n drawn from sizes, applied voltage
    U[-100, 100] mV and NaCl U[0.01, 0.5] M, each with its own charge seed."""
    pick = (splitmix64(substream(seed, 1), count) % np.uint64(len(sizes))).astype(np.int64)
    volts = uniform(substream(seed, 2), count, -0.1, 0.1)
    salt = uniform(substream(seed, 3), count, 0.01, 0.5)
    out = []
    for i in range(count):
        sp = [Species(+1, 0.95, float(salt[i]), "Na+"), Species(-1, 1.81, float(salt[i]), "Cl-"), WATER]
        out.append(channel_problem(int(sizes[pick[i]]), phi_hi_V=float(volts[i]), species=sp,
                                   charge_seed=substream(seed, 100 + i), name=f"batch_{i}"))
    return out


def request_stream(count: int = 2000, seed: int = 4, mean_gap_s: float = 0.005, n_lo: int = 49, n_hi: int = 193):
    """Poisson arrivals (exponential gaps) of channel problems with log-uniform edge n in
    [n_lo, n_hi], random pore radius U[4, 6] A, voltage U[-100, 100] mV and NaCl U[0.01, 0.5] M.
    Returns a list of (arrival_time_s, PFProblem) built lazily by calling the second item."""
    gaps = -mean_gap_s * np.log(1.0 - uniform(substream(seed, 1), count))
    t = np.cumsum(gaps)
    edge = np.rint(np.exp(uniform(substream(seed, 2), count, math.log(n_lo), math.log(n_hi)))).astype(int)
    volts = uniform(substream(seed, 3), count, -0.1, 0.1)
    salt = uniform(substream(seed, 4), count, 0.01, 0.5)
    prad = uniform(substream(seed, 5), count, 4.0, 6.0)
    reqs = []
    for i in range(count):
        def make(i=i):
            sp = [Species(+1, 0.95, float(salt[i]), "Na+"), Species(-1, 1.81, float(salt[i]), "Cl-"), WATER]
            return channel_problem(int(edge[i]), pores=((0.0, 0.0, float(prad[i])),), phi_hi_V=float(volts[i]),
                                   species=sp, charge_seed=substream(seed, 1000 + i), name=f"req_{i}")
        reqs.append((float(t[i]), int(edge[i]), make))
    return reqs
