"""CPU FP64 oracle for RI-HF energies and analytic gradients -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
product path never imports, links or executes anything here, and this package
shares no code with it (the only shared module is the seeded input generator
``paper_2407_19614_gb300.workloads``, which holds no method arithmetic).

Layout
  md_integrals.c  McMurchie-Davidson Gaussian integrals and first derivatives
                  (S, T, V, (P|Q), (mu nu|P), (mu nu|lambda sigma)), Boys function
                  in long double.
  integrals.py    ctypes binding of md_integrals.c (builds it with gcc on demand).
  basis.py        primitive and contraction normalisation, Cartesian -> real
                  solid-harmonic transform (closed form), AO bookkeeping.
  rihf.py         RI fitting, RI-J/RI-K Fock build, SCF with Pulay DIIS, energy,
                  analytic gradient (Eq. rihf_gradient), brute-force 4-centre HF.

Parity status per function is listed in the module docstrings; every function
here is pinned by ``tests/test_oracle_*.py`` (closed forms, invariances,
one-centre exactness, finite differences).
"""
