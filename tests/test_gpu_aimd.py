"""AIMD robustness of the SCF along the benchmark's own trajectory: (H2O)8
from its seeded start, velocity Verlet at 0.5 fs with the library's forces,
every step's SCF warm-started from the previous orbitals.

This trajectory heats quickly (the even-tempered basis gives forces near
1 Eh/bohr, atoms move by up to 4 bohr in 35 steps) and once made the
warm-started SCF stall near max|e| 7e-7 on both paths, at steps 34 to 36.  Here
every step of 40 must converge, the warm-started energy at the last geometry
must equal a cold start from the core Hamiltonian, and the FP64 path replaying
the same geometries must agree with the mixed path within the mixed tolerance.
"""
import copy

import numpy as np
import pytest

from paper_2407_19614_gb300 import workloads as W

pytestmark = pytest.mark.gpu
CONV = dict(conv_e=1e-8, conv_diis=1e-7, max_iter=60)
DT = 0.5 * W.FS_TO_AU


def _R():
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    return R


def _trajectory(R, precision, nsteps, replay=None):
    mol = W.water8(0)
    m = W.masses_au(mol.Z)[:, None]
    ctx = R.Context(mol, precision=precision, **CONV)
    x, v = mol.xyz.copy(), W.maxwell_boltzmann(mol.Z, 300.0, 0)
    ctx.scf(guess=0, outputs=False)
    g = ctx.gradient()
    geoms, E, F = [], [], []
    for k in range(nsteps):
        a = -g / m
        x = replay[k] if replay is not None else x + v * DT + 0.5 * a * DT * DT
        ctx.update_geometry(x)
        out = ctx.scf(guess=2, outputs=False)     # raises on NOT_CONVERGED
        gn = ctx.gradient()
        v = v + 0.5 * (a - gn / m) * DT
        g = gn
        geoms.append(x.copy())
        E.append(out["energy"])
        F.append(gn.copy())
    return ctx, geoms, np.array(E), F


def test_forty_warm_started_steps_converge_on_both_paths():
    R = _R()
    ctx, geoms, E, F = _trajectory(R, R.PRECISION_MIXED, 40)
    assert np.abs(geoms[-1] - geoms[0]).max() > 2.0          # the trajectory really moved
    mol = copy.copy(W.water8(0))
    mol.xyz = geoms[-1]
    cold = R.Context(mol, precision=R.PRECISION_MIXED, **CONV).scf(guess=0, outputs=False)
    assert abs(cold["energy"] - E[-1]) <= 1e-8
    ctx64, _, E64, F64 = _trajectory(R, R.PRECISION_FP64, 40, replay=geoms)
    assert np.abs(E - E64).max() <= 1e-6
    assert max(np.abs(a - b).max() for a, b in zip(F, F64)) <= 1e-5
