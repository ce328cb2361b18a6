"""GB300-native UGKWP wave-particle step (arXiv 2007.13091) behind a C-ABI.

The compute lives in the CUDA library ``libugkwp.so`` built from ``csrc/``;
``ugkwp`` is the thin ctypes binding with the C-ABI's names, and
``workloads`` generates the seeded synthetic meshes and states.
"""
