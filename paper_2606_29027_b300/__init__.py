"""B300-native SLAR + adaptive-weight implicit LoMaC for the Vlasov-Poisson system.

The compute path lives in the C-ABI shared library ``libslar.so`` (CUDA, sm_103a) built
from ``csrc/``; :mod:`paper_2606_29027_b300.slar` is a thin ctypes binding to it.
:mod:`paper_2606_29027_b300.inputs` generates the seeded synthetic workloads.
"""
