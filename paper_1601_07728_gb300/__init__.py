"""GB300-native core-excitation BSE hot path: H psi, Haydock, GMRES.

The compute path lives in the C-ABI library ``libbse.so`` (hand-written
sm_103a CUDA, sources under ``csrc/``); ``bse`` is its thin ctypes binding.
Importing this package does not load the library; ``bse.lib()`` does, and
raises if the library has not been built.
"""
__all__ = ["synth", "bse"]
