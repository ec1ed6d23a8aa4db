"""Schwarz screening of primary shell pairs (Sec. 3.1.1): Q_ab = sqrt(max (mu nu|mu nu))
from the GPU four-centre recursion against brute-force four-centre integrals of the
oracle; screened pairs vanish from (mu nu|P); a loose threshold changes the energy
by far less than it screens."""
import numpy as np
import pytest

from oracle import integrals as OI
from oracle import basis as OB
from oracle import rihf as O
from paper_2407_19614_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _R():
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    return R


def test_schwarz_factors_match_four_centre_diagonal():
    R = _R()
    mol = W.water_monomer(2)
    ctx = R.Context(mol)
    Q = ctx.matrix("SCHWARZ")
    bas = OB.AOBasis(mol.primary, mol.xyz)
    eri = OI.eri4(bas.cb)                       # Cartesian, same primitive normalisation
    offs = np.concatenate([[0], np.cumsum([(s.l + 1) * (s.l + 2) // 2 for s in mol.primary])])
    ns = len(mol.primary)
    for a in range(ns):
        for b in range(a + 1):
            ia = range(offs[a], offs[a + 1])
            ib = range(offs[b], offs[b + 1])
            d = max(eri[i, j, i, j] for i in ia for j in ib)
            assert Q[a * (a + 1) // 2 + b] == pytest.approx(np.sqrt(d), rel=1e-11)


def test_loose_threshold_screens_pairs_and_keeps_energy():
    R = _R()
    mol = W.water8(1)
    full = R.Context(mol, conv_e=1e-10, conv_diis=5e-9)    # default tau = 0
    kept_full, total = full.screening_stats()
    assert kept_full == total                   # the default keeps every pair
    e_full = full.scf()["energy"]
    # cond((P|Q)) ~ 1e9 for this auxiliary set: the fit amplifies even pairs with
    # (mu nu|mu nu) <= 1e-14 into micro-hartree energy changes
    tight = R.Context(mol, schwarz_tau=1e-14, conv_e=1e-10, conv_diis=5e-9)
    assert tight.screening_stats()[0] < total
    assert abs(tight.scf()["energy"] - e_full) < 1e-4
    loose = R.Context(mol, schwarz_tau=1e-7, conv_e=1e-10, conv_diis=5e-9)
    kept, total2 = loose.screening_stats()
    assert kept < total2
    Q = loose.matrix("SCHWARZ")
    T = loose.matrix("T3")
    # a dropped pair's block of (mu nu|P) is exactly zero
    dropped = [(a, b) for a in range(len(mol.primary)) for b in range(a + 1) if Q[a * (a + 1) // 2 + b] ** 2 <= 1e-7]
    assert dropped
    ao = np.concatenate([[0], np.cumsum([2 * s.l + 1 for s in mol.primary])])
    a, b = dropped[0]
    assert np.all(T[:, ao[a]:ao[a + 1], ao[b]:ao[b + 1]] == 0.0)
    # (no SCF at tau = 1e-7: with cond((P|Q)) ~ 1e9 the truncated integrals are
    # no longer consistent with the metric and the fitted Coulomb energy fails)
