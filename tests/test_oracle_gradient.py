"""Pins for the oracle's analytic RI-HF gradient (Eq. rihf_gradient).

* central finite differences of the oracle energy (5-point stencil);
* zero net force (translational invariance) and zero net torque (rotational
  invariance) for an isolated molecule;
* a planted mistake -- the 1/2 factors of Y and Z applied with plain C_occ
  instead of C~ = sqrt(2) C_occ -- is caught by the finite-difference test,
  which is what decides that reading of the paper.
"""
import numpy as np
import pytest

from oracle import rihf
from paper_2407_19614_gb300 import workloads as W


def _fd_gradient(mol, pure, h=2e-3, coords=None, conv=(1e-13, 1e-11)):
    g = np.zeros_like(mol.xyz)
    coords = coords or [(a, d) for a in range(mol.natoms) for d in range(3)]
    for a, d in coords:
        vals = []
        for s in (2 * h, h, -h, -2 * h):
            x = mol.xyz.copy()
            x[a, d] += s
            vals.append(rihf.energy_at(mol, x, pure=pure, conv_e=conv[0], conv_diis=conv[1]))
        g[a, d] = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
    return g


@pytest.fixture(scope="module")
def water_grad():
    mol = W.water_monomer(0)
    s = rihf.System(mol)
    r = rihf.rihf_energy(s, conv_e=1e-13, conv_diis=1e-11)
    return mol, s, r, rihf.rihf_gradient_terms(s, r)


def test_gradient_matches_finite_differences(water_grad):
    mol, s, r, g = water_grad
    fd = _fd_gradient(mol, True)
    assert np.abs(fd - g.grad).max() < 1e-8


def test_gradient_cartesian_basis_matches_finite_differences():
    mol = W.water_monomer(1)
    s = rihf.System(mol, pure=False)
    # Cartesian d shells on the auxiliary side make the metric nearly singular
    # (smallest eigenvalue ~1e-7), which puts the SCF noise floor near 1e-10
    # in the commutator; the step h = 4e-3 keeps the FD noise below 1e-8.
    r = rihf.rihf_energy(s, conv_e=1e-12, conv_diis=1e-9)
    g = rihf.rihf_gradient_terms(s, r)
    fd = _fd_gradient(mol, False, h=4e-3, coords=[(0, 0), (1, 2), (2, 1)], conv=(1e-12, 1e-9))
    for a, d in [(0, 0), (1, 2), (2, 1)]:
        assert abs(fd[a, d] - g.grad[a, d]) < 1e-8


def test_net_force_and_torque_vanish(water_grad):
    mol, s, r, g = water_grad
    assert np.abs(g.grad.sum(0)).max() < 1e-10
    torque = np.cross(mol.xyz, g.grad).sum(0)
    assert np.abs(torque).max() < 1e-9


def test_planted_orbital_scaling_mistake_is_caught(water_grad):
    """With C instead of C~ in Y and Z the gradient breaks the FD check."""
    mol, s, r, g = water_grad
    nocc = s.nocc
    C = r.C[:, :nocc]
    import scipy.linalg as sla
    cho = sla.cho_factor(s.A, lower=True)
    D = 2 * C @ C.T
    c = sla.cho_solve(cho, np.einsum("pmn,mn->p", s.T3, D))
    Tij = np.einsum("mi,pmn,nj->pij", C, s.T3, C)
    X = sla.cho_solve(cho, Tij.reshape(s.naux, -1)).reshape(Tij.shape)
    Y_bad = D[None] * c[:, None, None] - 0.5 * np.einsum("mi,pij,nj->pmn", C, X, C)
    # the 3-centre term alone moves by far more than the FD tolerance
    dT3 = s.eri3_ao(datom=1, ddim=2)
    good = np.sum(g.Y * dT3)
    bad = np.sum(Y_bad * dT3)
    assert abs(good - bad) > 1e-4
    assert abs(good - g.parts["three"][1, 2]) < 1e-12
