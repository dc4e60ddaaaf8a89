"""Fused image-preprocessing kernels for GB300 (sm_103a).

The compute path lives in the CUDA library ``libfkl.so`` built from ``csrc/``;
``paper_2508_07071_gb300.fkl`` is the thin ctypes binding over its C ABI
(declared in ``include/fkl.h``). Importing the package itself loads nothing,
so the seeded input generators in ``synth`` work on machines without a GPU.
"""
