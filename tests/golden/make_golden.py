"""Writes the stored expected values under tests/golden/ -- calls only oracle/.

    python tests/golden/make_golden.py

water8_seed0.json: FP64 oracle RI-HF energy, orbital energies and analytic
gradient of the (H2O)8 cluster (seed 0, 7 A cube, 192 primary / 848 auxiliary
spherical functions), converged to max|X^T(FDS-SDF)X| < 1e-9 and |dE| < 1e-11
(an SCF error e moves the forces by about e / gap times the orbital-response
coupling: re-converging from 5e-9 to 1e-9 moved these forces by 5.8e-8 Eh/bohr,
so a 1e-8 force comparison needs both sides near 1e-9).
The oracle is pinned by tests/test_oracle_*.py (closed forms, invariances,
one-centre exactness, finite differences); the paper prints no numeric example.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import rihf  # noqa: E402
from paper_2407_19614_gb300 import workloads as W  # noqa: E402

CONV = dict(conv_e=1e-11, conv_diis=1e-9, max_iter=300)


def main():
    mol = W.water8(0)
    t0 = time.time()
    s = rihf.System(mol)
    r = rihf.rihf_energy(s, **CONV)
    assert r.converged, "oracle SCF did not converge"
    g = rihf.rihf_gradient_terms(s, r)
    out = dict(
        workload="(H2O)8, seed 0, 7 A cube, even-tempered primary O 3s2p1d / H 2s1p (a0 0.1, ratio 3), "
                 "auxiliary O 8s6p4d2f / H 4s3p2d (a0 0.15, ratio 2.5), spherical",
        N=s.nao, Naux=s.naux, nocc=s.nocc, conv=CONV, iterations=r.iterations,
        energy=r.E, eps_occ=r.eps[: s.nocc].tolist(), grad=g.grad.tolist(),
        grad_parts={k: v.tolist() for k, v in g.parts.items()},
        oracle_seconds=time.time() - t0,
    )
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "water8_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, "E =", r.E)


if __name__ == "__main__":
    main()
