"""GB300-native RI-HF energies and analytic gradients (Stocks, Palethorpe, Barca,
"Multi-GPU RI-HF Energies and Analytic Gradients", Sec. 2-3).

The compute path lives in the CUDA library ``librihf.so`` built from ``csrc/``;
``rihf`` is a thin ctypes binding with the same entry-point names as the C ABI.
``workloads`` holds the seeded synthetic geometries and basis-set descriptions
(data only) that both the library and the independent CPU oracle consume.
Importing this package does not load the CUDA library; ``rihf.load()`` does.
"""

__all__ = ["workloads", "rihf"]
