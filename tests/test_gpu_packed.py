"""Pair-packed storage of the fitted tensor and its chunked expansion.

B (and the gradient's Y) live on the device as Naux x N(N+1)/2 pair-packed
FP64; RI-K and the gradient expand them chunk by chunk of auxiliary functions
(as many as the free memory holds; opt.aux_chunk caps the chunk).  With ragged
chunks of 7 auxiliary functions the energy and forces must equal those of the
unchunked run (same kernels, different chunking: the tensor-core products are
exact integer sums per output row, the FP64 ones differ in summation order
only) and the FP64 oracle's.
"""
import numpy as np
import pytest

from oracle import rihf as O
from paper_2407_19614_gb300 import workloads as W

pytestmark = pytest.mark.gpu
CONV = dict(conv_e=1e-10, conv_diis=1e-9, max_iter=100)


def _R():
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    return R


@pytest.fixture(scope="module")
def dimer_oracle():
    mol = W.water_n(2, 0)
    s = O.System(mol)
    r = O.rihf_energy(s, conv_e=1e-12, conv_diis=1e-10)
    return mol, r, O.rihf_gradient_terms(s, r)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_chunked_expansion_matches_whole_and_oracle(precision, dimer_oracle):
    R = _R()
    mol, r, g = dimer_oracle
    assert mol.aux and sum(2 * sh.l + 1 for sh in mol.aux) % 7 != 0   # a ragged last chunk
    whole = R.Context(mol, precision=precision, **CONV)
    ew = whole.scf(outputs=False)["energy"]
    gw = whole.gradient()
    chunked = R.Context(mol, precision=precision, aux_chunk=7, **CONV)
    ec = chunked.scf(outputs=False)["energy"]
    gc = chunked.gradient()
    assert abs(ec - ew) <= 1e-9
    assert np.abs(gc - gw).max() <= 1e-8
    tol_e, tol_f = (1e-9, 1e-8) if precision == 0 else (1e-6, 1e-5)
    assert abs(ec - r.E) <= tol_e
    assert np.abs(gc - g.grad).max() <= tol_f
    # a second SCF and gradient on the same geometry (the gradient used the
    # expansion buffer as scratch in between)
    assert abs(chunked.scf(guess=2, outputs=False)["energy"] - ec) <= 1e-9
    assert abs(whole.scf(guess=2, outputs=False)["energy"] - ew) <= 1e-9
    assert np.abs(whole.gradient() - gw).max() <= 1e-8
