"""GB300-native OPO split-step hot path (arXiv 2410.02532).

Submodules:
  ``opo``        ctypes binding of the C-ABI library ``libopo.so`` (the product path)
  ``workloads``  seeded synthetic inputs and workload presets
  ``build``      compiles ``libopo.so`` for sm_103a with nvcc

Importing the package does not load the CUDA library; ``opo.lib()`` does, and
raises if it has not been built.
"""
