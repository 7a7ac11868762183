"""GB300-native Wilson-clover Dirac operator and mixed-precision solvers.

The compute path is the C-ABI library ``liboq.so`` (hand-written sm_103a
CUDA); ``paper_2202_07388_gb300.oq`` is its thin ctypes binding.  The library
is loaded lazily, on first use, and loading fails loudly if it has not been
built: there is no CPU fallback.
"""
__all__ = ["synth"]
