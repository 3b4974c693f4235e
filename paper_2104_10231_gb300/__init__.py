"""GB300-native Relative Resolution (RelRes) Lennard-Jones molecular dynamics.

The compute path is a C-ABI shared library (``librelres.so``, CUDA for
sm_103a, declared in ``include/relres.h``); ``paper_2104_10231_gb300.relres``
is its thin ctypes binding.  ``systems`` builds seeded synthetic inputs.
Importing this package does not load the CUDA library.
"""
__all__ = ["systems", "relres"]
