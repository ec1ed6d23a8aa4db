"""The synthetic input recipe: function counts of the basis sets, cluster
geometry constraints and seeded reproducibility (the inputs stand in for the
paper's water-cluster workloads, Sec. 4)."""
import numpy as np

from paper_2407_19614_gb300 import workloads as W

ANG = 1.0 / 0.529177210903


def _nf(shells):
    return sum(2 * s.l + 1 for s in shells)


def test_function_counts():
    m = W.water_monomer(0)
    assert (_nf(m.primary), _nf(m.aux)) == (24, 106)
    m8 = W.water8(0)
    assert (_nf(m8.primary), _nf(m8.aux), m8.natoms) == (192, 848, 24)
    m16 = W.water16(0)
    assert (_nf(m16.primary), _nf(m16.aux)) == (384, 1696)
    big = W.make_molecule(2, 6.0, 0, "large")
    assert (_nf(big.primary), _nf(big.aux)) == (2 * 58, 2 * 170)


def test_cluster_geometry_and_seeds():
    m = W.water8(3)
    xyz = m.xyz / ANG
    oxy = xyz[0::3]
    d = np.linalg.norm(oxy[:, None] - oxy[None], axis=-1) + np.eye(8) * 1e9
    assert d.min() >= 2.7 - 6 * 0.02 * np.sqrt(2)      # placement bound, less the 0.02 A noise
    for i in range(8):                                  # each monomer keeps its shape up to the noise
        oh = np.linalg.norm(xyz[3 * i + 1:3 * i + 3] - xyz[3 * i], axis=-1)
        assert np.all(np.abs(oh - 0.96) < 0.2)
    assert np.array_equal(W.water8(3).xyz, m.xyz)
    assert not np.array_equal(W.water8(4).xyz, m.xyz)
    assert list(m.Z) == [8, 1, 1] * 8 and m.nelec == 80


def test_batch_sizes_are_seeded_and_in_range():
    a = W.batch_sizes(256, seed=1)
    assert np.array_equal(a, W.batch_sizes(256, seed=1))
    assert a.min() >= 3 and a.max() <= 20 and len(a) == 256
