"""Mixed-precision SCF (RI-K on the tensor cores from BF16 digit planes in the
SCF iterations, a confirmation build with FP64-class products -- 7 digits, or
FP64 on request -- to declare convergence) against the FP64 CPU oracle,
through the C ABI.

Tolerances: |dE| <= 1e-6 Eh and max |dF| <= 1e-5 Eh/bohr against the FP64
oracle; the precision ladder ends on a confirmation build, so the result is in
practice as close as the FP64 path.
"""
import json
import os

import numpy as np
import pytest

from oracle import rihf as O
from paper_2407_19614_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "water8_seed0.json")


def _R():
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    return R


def test_mixed_monomer_energy_gradient():
    R = _R()
    mol = W.water_monomer(0)
    s = O.System(mol)
    r = O.rihf_energy(s, conv_e=1e-12, conv_diis=1e-10)
    g = O.rihf_gradient_terms(s, r)
    ctx = R.Context(mol, precision=R.PRECISION_MIXED, conv_e=1e-10, conv_diis=1e-8, max_iter=100)
    out = ctx.scf()
    st = ctx.scf_stats()
    assert st["tc_builds"] >= 3 and st["confirm_builds"] >= 1 and st["fp64_builds"] == 0
    assert abs(out["energy"] - r.E) <= 1e-6
    grad = ctx.gradient()
    assert np.abs(grad - g.grad).max() <= 1e-5


def test_mixed_confirmation_on_fp64_build_agrees():
    # the same SCF with the FP64 confirmation build: the two confirmations
    # accept states that agree to far below the mixed tolerance
    R = _R()
    mol = W.water_monomer(0)
    kw = dict(precision=R.PRECISION_MIXED, conv_e=1e-10, conv_diis=1e-8, max_iter=100)
    e7 = R.Context(mol, **kw).scf()["energy"]
    ctx = R.Context(mol, confirm_fp64=1, **kw)
    e64 = ctx.scf()["energy"]
    st = ctx.scf_stats()
    assert st["fp64_builds"] >= 1 and st["confirm_builds"] == 0 and st["tc_builds"] >= 3
    assert abs(e7 - e64) <= 1e-8


def test_mixed_water8_against_golden_and_fp64_path():
    R = _R()
    mol = W.water8(0)
    gold = json.load(open(GOLDEN))
    ctx = R.Context(mol, precision=R.PRECISION_MIXED, conv_e=1e-10, conv_diis=5e-9, max_iter=100)
    out = ctx.scf()
    st = ctx.scf_stats()
    # most iterations run the ladder; a few 7-digit builds confirm convergence
    assert st["tc_builds"] >= 5 and st["fp64_builds"] == 0 and 1 <= st["confirm_builds"] <= 3
    assert abs(out["energy"] - gold["energy"]) <= 1e-6
    grad = ctx.gradient()
    assert np.abs(grad - np.array(gold["grad"])).max() <= 1e-5
    ctx64 = R.Context(mol, conv_e=1e-10, conv_diis=5e-9, max_iter=100)
    out64 = ctx64.scf()
    assert abs(out["energy"] - out64["energy"]) <= 1e-6


@pytest.mark.parametrize("digits", [5, 6, 7])
def test_mixed_fixed_digit_counts_converge(digits):
    # a fixed digit count: the 7-digit confirmation build accepts the SCF state
    # only when the ladder iterations already reached the FP64-class fixed point
    R = _R()
    mol = W.water_monomer(1)
    s = O.System(mol)
    r = O.rihf_energy(s, conv_e=1e-12, conv_diis=1e-10)
    ctx = R.Context(mol, precision=R.PRECISION_MIXED, mixed_digits=digits, conv_e=1e-10, conv_diis=1e-8,
                    max_iter=100)
    out = ctx.scf()
    st = ctx.scf_stats()
    assert st["tc_builds"] >= 3
    assert abs(out["energy"] - r.E) <= 1e-6


def test_tensor_core_fit_matches_fp64_fit():
    # B = L^{-1} T with the rank-64 updates on the tensor cores (7 digits) against
    # the FP64 substitution: the digits carry 55 bits of each row's largest
    # element per 64-column block, so the two solves agree to near FP64
    # rounding even through cond(L) ~ 5e4
    R = _R()
    mol = W.water8(0)
    b64 = R.Context(mol).matrix("B")
    bmx = R.Context(mol, precision=R.PRECISION_MIXED).matrix("B")
    N = b64.shape[1]
    il = np.tril_indices(N)
    d = np.abs(bmx[:, il[0], il[1]] - b64[:, il[0], il[1]]).max()
    scale = np.abs(b64).max()
    print("\nmax |B_tc - B_fp64| = %.3e (max |B| = %.3e)" % (d, scale))
    assert d <= 1e-10 * scale
