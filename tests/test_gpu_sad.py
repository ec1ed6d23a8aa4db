"""SAD cold start (guess 5): superposition of atomic densities.

The library runs one RI-HF SCF per atom type of the isolated, spherically
averaged atom (fractional occupations of the ground configuration, every Fock
matrix averaged over rotations, orbitals occupied by angular momentum) and
places the atoms' densities on their basis-function blocks; the first SCF
iteration builds J from D_SAD and K from its factor (the density form of RI-K,
Eq. k_ri_1, since D_SAD is not idempotent and has more columns than occupied
orbitals: O 1s 2s 2p, H 1s give seven per water against five occupied).

Parity: D_SAD element by element against the oracle's superposition of the
same atomic SCFs (both converged to max|e| <= 1e-7, so 1e-6 on D).  Then the
converged SCF from the SAD start equals the one from the core Hamiltonian.
"""
import numpy as np
import pytest

from oracle import rihf as O
from paper_2407_19614_gb300 import workloads as W

pytestmark = pytest.mark.gpu
CONV = dict(conv_e=1e-10, conv_diis=1e-9, max_iter=100)
CONFIG = {"O": ([2.0, 2.0, 4 / 3, 4 / 3, 4 / 3], [0, 0, 1, 1, 1]), "H": ([1.0], [0])}


def _R():
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    return R


def _oracle_sad(mol, basis):
    counts_p = W.PRIMARY_SMALL if basis == "small" else W.PRIMARY_LARGE
    counts_a = W.AUX_SMALL if basis == "small" else W.AUX_LARGE
    syms = {1: "H", 8: "O"}
    dens = {}
    for sym in ("O", "H"):
        atom = W.Molecule(Z=np.array([W.Z_OF[sym]], dtype=np.int32), xyz=np.zeros((1, 3)),
                          primary=W.even_tempered([sym], counts_p, W.PRIMARY_A0, W.PRIMARY_RATIO),
                          aux=W.even_tempered([sym], counts_a, W.AUX_A0, W.AUX_RATIO))
        s = O.System(atom)
        occ, occ_l = CONFIG[sym]
        r = O.rihf_energy(s, occ=occ, occ_l=occ_l, sph=O.sph_labels(atom.primary), conv_e=1e-12, conv_diis=1e-9,
                          max_iter=300)
        assert r.converged
        dens[sym] = r.D
    blocks = [dens[syms[int(z)]] for z in mol.Z]
    N = sum(b.shape[0] for b in blocks)
    D = np.zeros((N, N))
    o = 0
    for b in blocks:
        D[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    return D


@pytest.mark.parametrize("basis,mol", [("small", W.water_n(2, 0)), ("large", W.water_monomer(2))],
                         ids=["dimer-small", "monomer-large"])
def test_sad_density_against_oracle(basis, mol):
    R = _R()
    if basis == "large":
        mol = W.make_molecule(1, 0.0, 2, "large")
    ctx = R.Context(mol, **CONV)
    ctx.scf(guess=5, outputs=False)
    D = ctx.matrix("DSAD")
    Do = _oracle_sad(mol, basis)
    assert D.shape == Do.shape
    print("\nmax |D_SAD - oracle| = %.2e (max %.2e)" % (np.abs(D - Do).max(), np.abs(Do).max()))
    assert np.abs(D - Do).max() <= 1e-6


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_sad_start_converges_to_the_core_start_solution(precision):
    R = _R()
    mol = W.water8(0)
    kw = dict(precision=precision, conv_e=1e-10, conv_diis=5e-9, max_iter=100)
    a = R.Context(mol, **kw)
    oa = a.scf(guess=0, outputs=False)
    b = R.Context(mol, **kw)
    ob = b.scf(guess=5, outputs=False)
    assert b.learn_stats()["last_guess"] == 5
    assert abs(oa["energy"] - ob["energy"]) <= 1e-9
    print("\nSCF iterations: core start %d, SAD start %d" % (oa["iterations"], ob["iterations"]))
    assert ob["iterations"] < oa["iterations"]
    # two SCFs converged independently to max|e| < 5e-9: forces are first order
    # in the density error, so they agree to a few 1e-8
    assert np.abs(a.gradient() - b.gradient()).max() <= 5e-8
