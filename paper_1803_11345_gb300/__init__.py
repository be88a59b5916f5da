"""GB300-native hybrid central-moment / BGK lattice Boltzmann solver for the coupled
Cahn-Hilliard--Navier-Stokes equations (De Rosis, Saito, Kaneko & Abe, arXiv:1803.11345).

The hot path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI); ``lbm`` is the thin ctypes
binding.  Importing this package does not load the CUDA library: import ``lbm`` for that.
"""
