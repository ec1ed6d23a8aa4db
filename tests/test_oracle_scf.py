"""Pins for the oracle's RI fitting, Fock build and SCF (Sec. 2.2 of the paper).

* converged density: (D/2) S (D/2) = D/2, Tr DS = n_elec, F C = S C eps;
* the energy is invariant under rigid rotation and translation;
* one-centre exactness: for an atom whose auxiliary set spans every product of
  primary functions, RI-HF equals brute-force four-centre HF (Eq. ri_eri is exact);
* RI-HF approaches four-centre HF as the auxiliary set grows, and for a fixed
  density the fitted Coulomb energy never exceeds the exact one (the Coulomb
  metric makes the fit variational: E_J - E_J^RI = 1/2 (rho - rho~|rho - rho~) >= 0);
* Eq. k_ri_1 (density form) and Eqs. k_ri_2/tp (occupied-orbital form) agree.
"""
import copy
import math

import numpy as np
import pytest

from oracle import rihf
from paper_2407_19614_gb300 import workloads as W


@pytest.fixture(scope="module")
def water():
    s = rihf.System(W.water_monomer(0))
    return s, rihf.rihf_energy(s)


def test_converged_density_properties(water):
    s, r = water
    assert r.converged
    Dh = r.D / 2
    assert np.abs(Dh @ s.S @ Dh - Dh).max() < 1e-9
    assert np.sum(r.D * s.S) == pytest.approx(s.Z.sum(), abs=1e-9)
    FC = r.F @ r.C
    SCe = s.S @ r.C @ np.diag(r.eps)
    assert np.abs(FC - SCe)[:, : s.nocc].max() < 1e-8
    assert r.eps[s.nocc] > r.eps[s.nocc - 1]      # closed-shell aufbau with a gap


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_energy_rigid_motion_invariance(water):
    s, r = water
    mol = W.water_monomer(0)
    xyz = mol.xyz @ _rot([1, 2, -0.5], 0.77).T + np.array([1.5, -0.3, 2.2])
    assert rihf.energy_at(mol, xyz) == pytest.approx(r.E, abs=1e-10)


def test_k_density_form_equals_orbital_form(water):
    s, r = water
    L, B = rihf.cholesky_fit(s.A, s.T3)
    Co = r.C[:, : s.nocc]
    K1 = rihf.exchange_density_ri(B, rihf.density(Co))
    K2 = rihf.exchange_ri(B, Co)
    assert np.abs(K1 - K2).max() < 1e-12


def test_fitted_factor_reproduces_metric(water):
    s, r = water
    L, B = rihf.cholesky_fit(s.A, s.T3)
    assert np.abs(L @ L.T - s.A).max() < 1e-12
    # sum_P B^P B^P == T^T A^{-1} T  (Eq. symmetric_ri)
    naux = s.naux
    T = s.T3.reshape(naux, -1)
    Bf = B.reshape(naux, -1)
    lhs = Bf.T @ Bf
    rhs = T.T @ np.linalg.solve(s.A, T)
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(rhs).max()


@pytest.mark.parametrize("Z,nprim,pure,aux_lmax", [(2, (4,), True, 0), (4, (4, 2), False, 2)])
def test_one_centre_exactness(Z, nprim, pure, aux_lmax):
    mol = W.tiny_atom_basis(Z=Z, a0=0.4, ratio=3.0, nprim=nprim, aux_lmax=aux_lmax)
    s = rihf.System(mol, pure=pure)
    e_ri = rihf.rihf_energy(s).E
    e_4c = rihf.hf4c_energy(s).E
    assert e_ri == pytest.approx(e_4c, abs=2e-9)


def _water_with_aux(counts, a0, ratio, seed=2):
    mol = W.water_monomer(seed)
    sym = ["O", "H", "H"]
    mol = copy.copy(mol)
    mol.aux = W.even_tempered(sym, counts, a0, ratio)
    return mol


def test_ri_converges_to_four_centre_hf_and_coulomb_fit_is_variational():
    base = W.water_monomer(2)
    s4 = rihf.System(base)
    r4 = rihf.hf4c_energy(s4)
    errs = []
    for counts, a0, ratio in [({"O": (3, 2, 1), "H": (2, 1)}, 0.2, 3.0),
                              ({"O": (8, 6, 4, 2), "H": (4, 3, 2)}, 0.15, 2.5),
                              ({"O": (12, 10, 8, 5, 2), "H": (8, 6, 4, 2)}, 0.12, 1.9)]:
        s = rihf.System(_water_with_aux(counts, a0, ratio))
        r = rihf.rihf_energy(s)
        errs.append(abs(r.E - r4.E))
        # Coulomb energy with the converged four-centre density, fitted vs exact
        L, B = rihf.cholesky_fit(s.A, s.T3)
        ej_ri = 0.5 * np.sum(r4.D * rihf.coulomb_ri(B, r4.D))
        ej = 0.5 * np.einsum("mn,mnls,ls->", r4.D, r4.eri, r4.D)
        assert ej_ri <= ej + 1e-12
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3
