"""Batched AIMD steps over independent molecules (concurrent contexts) and
CUDA-graph replay of the SCF iterations: both must reproduce the results of
the plain per-molecule path (same kernels; FP64 atomics make the last bits
order-dependent, hence the 1e-9 / 1e-8 bounds)."""
import numpy as np
import pytest

from paper_2407_19614_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _R():
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    return R


MOLS = [W.water_monomer(0), W.water_n(2, 0), W.water_n(3, 1), W.water_n(4, 2)]
CONV = dict(conv_e=1e-10, conv_diis=1e-9, max_iter=100)


def _displaced(mol, seed):
    rng = np.random.default_rng(seed)
    return mol.xyz + 0.02 * rng.standard_normal(mol.xyz.shape)


@pytest.mark.parametrize("nthreads", [1, 0])
def test_batch_step_matches_individual_contexts(nthreads):
    R = _R()
    batch = [R.Context(m, **CONV) for m in MOLS]
    single = [R.Context(m, **CONV) for m in MOLS]
    for c in batch + single:
        c.scf(guess=0, outputs=False)
    xs = [_displaced(m, i) for i, m in enumerate(MOLS)]
    E, G, it = R.batch_step(batch, xs, guess=2, nthreads=nthreads)
    for i, (c, x) in enumerate(zip(single, xs)):
        c.update_geometry(x)
        out = c.scf(guess=2, outputs=False)
        g = c.gradient()
        assert abs(E[i] - out["energy"]) <= 1e-9
        assert np.abs(G[i] - g).max() <= 1e-8
        assert it[i] >= 1


def test_batch_step_without_new_geometry_and_errors():
    R = _R()
    ctxs = [R.Context(m, **CONV) for m in MOLS[:2]]
    for c in ctxs:
        c.scf(guess=0, outputs=False)
    E, G, it = R.batch_step(ctxs, None, guess=2)
    assert np.all(np.isfinite(E)) and G[1].shape == (MOLS[1].natoms, 3)
    # a context that cannot run its gradient (no converged SCF) makes the
    # batch report that molecule's error
    fresh = R.Context(MOLS[0], max_iter=1, conv_e=1e-14, conv_diis=1e-14)
    with pytest.raises(R.RihfError) as e:
        R.batch_step([ctxs[0], fresh], None, guess=0)
    assert "molecule 1" in str(e.value)


@pytest.mark.parametrize("precision", [0, 1])
def test_cuda_graph_replay_matches_eager(precision):
    R = _R()
    mol = W.water_n(3, 0)
    res = []
    for graphs in (0, 1):
        c = R.Context(mol, precision=precision, cuda_graphs=graphs, **CONV)
        out0 = c.scf(guess=0, outputs=False)
        c.update_geometry(_displaced(mol, 7))
        out1 = c.scf(guess=2, outputs=False)
        res.append((out0["energy"], out1["energy"], out0["iterations"], out1["iterations"], c.gradient()))
    a, b = res
    assert abs(a[0] - b[0]) <= 1e-9 and abs(a[1] - b[1]) <= 1e-9
    assert np.abs(a[4] - b[4]).max() <= 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_against_the_oracle(precision):
    """Every molecule of a batch step against the FP64 CPU oracle at its new
    geometry: FP64 within 1e-9 Eh / 1e-8 Eh/bohr, mixed within 1e-6 / 1e-5."""
    import copy

    from oracle import rihf as O
    R = _R()
    mols = MOLS[:3]
    ctxs = [R.Context(m, precision=precision, **CONV) for m in mols]
    for c in ctxs:
        c.scf(guess=0, outputs=False)
    xs = [_displaced(m, 10 + i) for i, m in enumerate(mols)]
    E, G, it = R.batch_step(ctxs, xs, guess=2)
    tol_e, tol_f = (1e-9, 1e-8) if precision == 0 else (1e-6, 1e-5)
    for i, (m, x) in enumerate(zip(mols, xs)):
        mk = copy.copy(m)
        mk.xyz = x
        s = O.System(mk)
        r = O.rihf_energy(s, conv_e=1e-12, conv_diis=1e-10)
        g = O.rihf_gradient_terms(s, r)
        assert abs(E[i] - r.E) <= tol_e, (i, E[i] - r.E)
        assert np.abs(G[i] - g.grad).max() <= tol_f, i
