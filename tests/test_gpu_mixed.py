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


def _k_digit_bound(B, Co, digits):
    """Bound of |K_tc - K| for K = -sum_P (B^P C)(B^P C)^T built as on the
    tensor cores: H = B C~ (C~ = sqrt(2) C_occ) from `digits` balanced 8-bit
    digits of the rows of B and of C~ (every element keeps 7 + 8(digits - 1)
    bits below its row's largest exponent; the dropped digit pairs weigh less
    than that, constant 8 as for the plain GEMM), then K = -1/2 H H^T from
    digits of H's rows with the same rule over the whole (P, i) axis.  First
    order in the two errors."""
    naux, n, _ = B.shape
    bits = min(7 + 8 * (digits - 1), 55)
    u = 8.0 * 2.0 ** (-bits)
    Ct = np.sqrt(2.0) * Co
    H = np.einsum("pmn,ni->mpi", B, Ct).reshape(n, -1)         # rows mu, columns (P, i)
    bmax = np.abs(B).max(axis=2)                                 # max over nu of row (P, mu)
    cmax = np.abs(Ct).max(axis=0)                                # max over nu of column i of C~
    dH = u * n * np.einsum("pm,i->mpi", bmax, cmax).reshape(n, -1)
    hmax = np.abs(H).max(axis=1)
    prop = np.abs(H) @ dH.T
    return 0.5 * (prop + prop.T + u * H.shape[1] * np.outer(hmax, hmax))


@pytest.mark.parametrize("digits", [5, 6, 7])
def test_mixed_exchange_elementwise_per_digit_count(digits):
    """One tensor-core RI-K build (Eqs. k_ri_2 and tp) from the oracle's
    converged orbitals, element by element against the oracle's FP64 K of the
    same orbitals, inside the digit bound plus the FP64 fit's own 1e-11."""
    R = _R()
    mol = W.water_n(2, 0)
    s = O.System(mol)
    r = O.rihf_energy(s, conv_e=1e-12, conv_diis=1e-9)
    L, B = O.cholesky_fit(s.A, s.T3)
    Co = r.C[:, : s.nocc]
    Kref = O.exchange_ri(B, Co)
    ctx = R.Context(mol, precision=R.PRECISION_MIXED, mixed_digits=digits, max_iter=1, conv_e=1e-14,
                    conv_diis=1e-14)
    ctx.scf(guess=1, C_guess=r.C, outputs=False, allow_unconverged=True)
    assert ctx.scf_stats()["tc_builds"] == 1
    K = ctx.matrix("K")
    err = np.abs(K - Kref)
    bound = _k_digit_bound(B, Co, digits) + 1e-11 * max(1.0, np.abs(Kref).max())
    print("\n%d digits: max |K_tc - K| = %.3e, min slack %.3e" % (digits, err.max(), (bound - err).min()))
    assert np.all(err <= bound)
    assert np.abs(K - K.T).max() == 0.0
