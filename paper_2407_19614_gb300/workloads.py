"""Seeded synthetic workloads: water-cluster geometries and even-tempered basis sets.

This module is data only.  It draws random geometries and lists shell exponents;
it holds none of the RI-HF arithmetic (no normalisation, no integrals).  Both the
CUDA library and the CPU oracle consume its output, each applying its own
normalisation and transforms.

The workloads stand in for the paper's water-cluster benchmarks (Sec. 4,
Table "tab:timings": (H2O)10..60 with def2 basis sets).  The named basis sets and
the Supporting-Information geometries are not available, so:

* basis sets are even-tempered, uncontracted Gaussians: for every element and
  every angular momentum l with n_l shells the exponents are a0 * ratio**k,
  k = 0..n_l-1, chosen independently per l;
* clusters place oxygens uniformly at random in a cube (rejection sampling with
  a minimum O-O distance), attach hydrogens in the gas-phase water geometry
  under a uniformly random rotation (unit quaternion, Shoemake 1992), and add
  seeded Gaussian noise to every coordinate.

Coordinates are returned in bohr (1 bohr = 0.529177210903 Angstrom).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903
Z_OF = {"H": 1, "O": 8}

# Water monomer: O-H 0.96 Angstrom, H-O-H 104.5 degrees, H in the xz plane.
R_OH = 0.96
HALF_ANGLE = math.radians(104.5 / 2.0)


@dataclass
class Shell:
    """One contracted Cartesian/spherical Gaussian shell (unnormalised coefficients)."""

    atom: int
    l: int
    exps: list
    coefs: list


@dataclass
class Molecule:
    Z: np.ndarray            # (natoms,) int32 atomic numbers
    xyz: np.ndarray          # (natoms, 3) float64, bohr
    primary: list = field(default_factory=list)   # list[Shell]
    aux: list = field(default_factory=list)       # list[Shell]
    name: str = ""

    @property
    def natoms(self) -> int:
        return int(self.Z.shape[0])

    @property
    def nelec(self) -> int:
        return int(self.Z.sum())


# Shell counts per element and angular momentum (s, p, d, f, g).
PRIMARY_SMALL = {"O": (3, 2, 1), "H": (2, 1)}            # 24 spherical functions / water
AUX_SMALL = {"O": (8, 6, 4, 2), "H": (4, 3, 2)}          # 106 spherical functions / water
PRIMARY_LARGE = {"O": (4, 3, 2, 1), "H": (3, 2, 1)}      # 58 spherical functions / water
AUX_LARGE = {"O": (11, 8, 6, 3, 2), "H": (6, 4, 3)}      # 170 spherical functions / water

PRIMARY_A0, PRIMARY_RATIO = 0.1, 3.0
AUX_A0, AUX_RATIO = 0.15, 2.5


def even_tempered(symbols, counts, a0, ratio):
    """Uncontracted even-tempered shells for every atom, ordered atom-major then l."""
    shells = []
    for ia, sym in enumerate(symbols):
        for l, n in enumerate(counts[sym]):
            for k in range(n):
                shells.append(Shell(ia, l, [a0 * ratio ** k], [1.0]))
    return shells


def _random_rotation(rng):
    """Uniform random rotation matrix from a unit quaternion (Shoemake's method)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([
        math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
        math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
        math.sqrt(u1) * math.sin(2 * math.pi * u3),
        math.sqrt(u1) * math.cos(2 * math.pi * u3),
    ])
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _monomer_angstrom():
    s, c = math.sin(HALF_ANGLE), math.cos(HALF_ANGLE)
    return np.array([[0.0, 0.0, 0.0], [R_OH * s, 0.0, R_OH * c], [-R_OH * s, 0.0, R_OH * c]])


def water_cluster_angstrom(nwater, box, seed, min_oo=2.7, min_inter=1.5, noise=0.02):
    """(3*nwater, 3) Angstrom coordinates ordered O,H,H per molecule, and symbols."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mono = _monomer_angstrom()
    if nwater == 1:
        xyz = mono.copy()
    else:
        placed = []
        tries = 0
        while len(placed) < nwater:
            tries += 1
            if tries > 200000:
                raise RuntimeError("could not place %d waters in a %.2f A box" % (nwater, box))
            o = rng.random(3) * box
            rot = _random_rotation(rng)
            mol = o + mono @ rot.T
            ok = True
            for prev in placed:
                if np.linalg.norm(prev[0] - o) < min_oo:
                    ok = False
                    break
                d = np.linalg.norm(prev[:, None, :] - mol[None, :, :], axis=-1)
                if d.min() < min_inter:
                    ok = False
                    break
            if ok:
                placed.append(mol)
        xyz = np.concatenate(placed, axis=0)
    xyz = xyz + rng.normal(0.0, noise, size=xyz.shape)
    symbols = ["O", "H", "H"] * nwater
    return xyz, symbols


def make_molecule(nwater, box, seed, basis="small", name=""):
    xyz_a, symbols = water_cluster_angstrom(nwater, box, seed)
    prim_counts, aux_counts = (PRIMARY_SMALL, AUX_SMALL) if basis == "small" else (PRIMARY_LARGE, AUX_LARGE)
    return Molecule(
        Z=np.array([Z_OF[s] for s in symbols], dtype=np.int32),
        xyz=np.ascontiguousarray(xyz_a * ANGSTROM_TO_BOHR, dtype=np.float64),
        primary=even_tempered(symbols, prim_counts, PRIMARY_A0, PRIMARY_RATIO),
        aux=even_tempered(symbols, aux_counts, AUX_A0, AUX_RATIO),
        name=name or "(H2O)%d/%s/seed%d" % (nwater, basis, seed),
    )


def water_monomer(seed=0):
    """Single water with sigma = 0.02 A noise: 24 primary / 106 auxiliary functions."""
    return make_molecule(1, 0.0, seed, "small", "H2O/seed%d" % seed)


def water8(seed=0):
    """(H2O)8 in a 7 A cube: 192 primary / 848 auxiliary spherical functions."""
    return make_molecule(8, 7.0, seed, "small")


def water16(seed=0):
    """(H2O)16 in a 7*(16/8)^(1/3) A cube: 384 primary / 1696 auxiliary functions."""
    return make_molecule(16, 7.0 * (16 / 8) ** (1 / 3), seed, "small")


def water32_large(seed=0):
    """(H2O)32 in an 11 A cube with the larger basis: 1856 primary / 5440 auxiliary."""
    return make_molecule(32, 11.0, seed, "large")


def water_n(n, seed=0, basis="small"):
    """(H2O)n in a cube of side 7*(n/8)^(1/3) A."""
    return make_molecule(n, 7.0 * (n / 8.0) ** (1.0 / 3.0), seed, basis)


def batch_sizes(count=256, seed=0, lo=3, hi=20):
    """Cluster sizes n ~ U{lo..hi} for a batch of independent geometries."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=count)


AMU_TO_ME = 1822.888486
FS_TO_AU = 41.341374575751
KB_HARTREE = 3.166811563e-6
MASS_AMU = {1: 1.008, 8: 15.999}


def masses_au(Z):
    """Nuclear masses (electron masses) for atomic numbers Z."""
    return np.array([MASS_AMU[int(z)] * AMU_TO_ME for z in Z])


def maxwell_boltzmann(Z, temperature=300.0, seed=0):
    """Seeded Maxwell-Boltzmann velocities (bohr per atomic time unit) with the
    centre-of-mass momentum removed."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    m = masses_au(Z)
    v = rng.normal(size=(len(m), 3)) * np.sqrt(KB_HARTREE * temperature / m)[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v


def tiny_atom_basis(Z=2, a0=0.5, ratio=3.0, nprim=(3,), aux_lmax=None):
    """Single atom at the origin with an even-tempered primary set and, when
    ``aux_lmax`` is given, an auxiliary set holding every pair-sum exponent
    a_i + a_j for l = 0..aux_lmax (used for the one-centre exactness check)."""
    prim = []
    for l, n in enumerate(nprim):
        for k in range(n):
            prim.append(Shell(0, l, [a0 * ratio ** k], [1.0]))
    aux = []
    if aux_lmax is not None:
        by_l = {}
        for s in prim:
            by_l.setdefault(s.l, []).append(s.exps[0])
        for L in range(aux_lmax + 1):
            sums = set()
            for la, ea in by_l.items():
                for lb, eb in by_l.items():
                    if la + lb >= L and (la + lb - L) % 2 == 0:
                        for x in ea:
                            for y in eb:
                                sums.add(round(x + y, 12))
            for e in sorted(sums):
                aux.append(Shell(0, L, [e], [1.0]))
    return Molecule(Z=np.array([Z], dtype=np.int32), xyz=np.zeros((1, 3)), primary=prim, aux=aux,
                    name="atom Z=%d" % Z)
