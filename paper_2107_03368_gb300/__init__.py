"""GB300-native weighted-Hamming nearest-neighbour search over QUICCI
descriptors (arXiv 2107.03368): brute force, Dissimilarity Tree build and
query, and per-object voting, as hand-written sm_103a CUDA behind the C ABI
of include/dt.h.

Submodules:
  dt      the Python binding of libdt.so (same names as the C entry points)
  synth   seeded synthetic inputs shaped like the paper's workloads
"""

__all__ = ["dt", "synth"]
