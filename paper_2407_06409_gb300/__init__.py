"""GB300-native lMBD (linear-scaling many-body dispersion, arXiv 2407.06409).

The compute path is a C-ABI shared library of hand-written sm_103a CUDA kernels
(``csrc/``); ``lmbd`` is its thin ctypes binding.  ``inputs`` draws seeded
synthetic structures.
"""
