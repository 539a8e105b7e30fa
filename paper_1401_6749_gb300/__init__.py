"""GB300-native stochastic disconnected loops for twisted-mass fermions (arXiv:1401.6749).

The compute path is the C-ABI library ``libtmloops.so`` built from ``csrc/``
(hand-written sm_103a CUDA kernels); ``tmloops`` is its thin ctypes binding.
Importing this package does not load the library; ``tmloops`` does, and fails
loudly if the library is missing.
"""

__all__ = ["synth", "tmloops", "build"]
