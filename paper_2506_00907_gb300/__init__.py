"""GB300-native (sm_103a) lattice-Boltzmann solver with the moment-conserving
wall-link boundary schemes of Li, Chan, Feng & Wang (arXiv 2506.00907).

The compute path is the C-ABI library ``liblbm_gb300.so`` (hand-written CUDA,
declared in include/lbm.h); ``lbm`` is its thin ctypes binding.  Importing this
package loads nothing; the library is loaded on first use and there is no CPU
fallback.
"""
__all__ = ["lbm", "build", "inputs", "cases"]
