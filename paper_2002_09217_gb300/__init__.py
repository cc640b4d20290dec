"""GB300-native (sm_103a) time step of the two-population Particles-on-Demand
kinetic model of a van der Waals fluid (arXiv:2002.09217).

The step runs in hand-written CUDA kernels behind the C ABI of ``libpond``
(``include/pond.h``); ``paper_2002_09217_gb300.pond`` is the thin ctypes binding.
Importing the package does not load the CUDA library.
"""
__all__ = ["inputs"]
