"""GB300-native parameter-grid direct Monte Carlo (arXiv:1910.01965).

The compute path is the C-ABI library ``libzmc.so`` (hand-written CUDA for
sm_103a); ``zmc`` is its thin ctypes binding.  ``workloads`` builds seeded
synthetic inputs.  Importing the package loads nothing; the binding loads the
library on first use and raises if it is missing.
"""
__all__ = ["zmc", "workloads"]
