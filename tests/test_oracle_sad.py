"""Pins for the oracle's fractional-occupation SCF, the reference of the SAD
guess (superposition of atomic densities; the paper's cold start, Sec. 2.2).

The spherically averaged atom (1s2 2s2 2p4 for O, the four 2p electrons shared
evenly by the three 2p orbitals; 1s1 for H) has a spherically symmetric
density.  In a basis of real solid harmonics that fixes the structure of D
exactly: no coupling between different l or different m, and the same radial
block for every m of one l.  Aufbau with fractional occupations alone settles
in a symmetry-broken state (2p levels split 1 + 2 for the small basis), so the
atom's SCF averages every Fock matrix over rotations (exact for a spherical
density) and occupies its orbitals by angular momentum as the configuration
says (the small basis puts the 2p level below 2s); these tests check that the
fixed point is spherical and holds Z electrons.  The electron count Tr(D S) = Z and the
closed-shell limit (all n_i = 2 reproduces the plain SCF) pin the occupation
weights.
"""
import numpy as np
import pytest

from oracle import rihf as O
from paper_2407_19614_gb300 import workloads as W


def _atom(sym, basis):
    counts_p = W.PRIMARY_SMALL if basis == "small" else W.PRIMARY_LARGE
    counts_a = W.AUX_SMALL if basis == "small" else W.AUX_LARGE
    return W.Molecule(Z=np.array([W.Z_OF[sym]], dtype=np.int32), xyz=np.zeros((1, 3)),
                      primary=W.even_tempered([sym], counts_p, W.PRIMARY_A0, W.PRIMARY_RATIO),
                      aux=W.even_tempered([sym], counts_a, W.AUX_A0, W.AUX_RATIO))


def _atom_scf(sym, basis, occ, occ_l):
    s = O.System(_atom(sym, basis))
    r = O.rihf_energy(s, occ=occ, occ_l=occ_l, sph=O.sph_labels(s.mol.primary), conv_e=1e-12, conv_diis=1e-9,
                      max_iter=300)
    return s, r


@pytest.mark.parametrize("basis", ["small", "large"])
def test_oxygen_fractional_density_is_spherical(basis):
    s, r = _atom_scf("O", basis, [2.0, 2.0, 4 / 3, 4 / 3, 4 / 3], [0, 0, 1, 1, 1])
    assert r.converged
    assert abs(np.sum(r.D * s.S) - 8.0) < 1e-10
    # function labels (l, m) in the AO order of the spherical basis
    lm = [(sh.l, m) for sh in s.mol.primary for m in range(2 * sh.l + 1)]
    D = r.D
    for i, (li, mi) in enumerate(lm):
        for j, (lj, mj) in enumerate(lm):
            if li != lj or mi != mj:
                assert abs(D[i, j]) < 1e-8, (i, j)
    # the same radial block for every m of one l
    for l in range(max(x for x, _ in lm) + 1):
        blocks = []
        for m in range(2 * l + 1):
            idx = [i for i, (li, mi) in enumerate(lm) if li == l and mi == m]
            blocks.append(D[np.ix_(idx, idx)])
        for b in blocks[1:]:
            assert np.abs(b - blocks[0]).max() < 1e-8


def test_hydrogen_one_electron_and_closed_shell_limit():
    s, r = _atom_scf("H", "small", [1.0], [0])
    assert r.converged and abs(np.sum(r.D * s.S) - 1.0) < 1e-12
    # all n_i = 2 is the closed-shell SCF itself
    w = O.System(W.water_monomer(0))
    a = O.rihf_energy(w, conv_e=1e-12, conv_diis=1e-10)
    b = O.rihf_energy(w, occ=[2.0] * w.nocc, conv_e=1e-12, conv_diis=1e-10)
    assert abs(a.E - b.E) < 1e-12 and np.abs(a.D - b.D).max() < 1e-10
