"""GB300-native pseudospectral Navier-Stokes right-hand side (arXiv:1808.01309).

The compute path is the CUDA shared library ``libps.so`` built from ``csrc/``;
:mod:`paper_1808_01309_gb300.ps` is its thin ctypes binding.
"""
