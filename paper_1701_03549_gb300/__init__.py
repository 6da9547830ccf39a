"""GB300-native batched stochastic fire-spread simulation (arXiv:1701.03549).

The compute path is the CUDA library libfire (C ABI in include/fire.h, sources
in csrc/); ``fire`` is its thin Python binding and ``synth`` the seeded
synthetic-landscape generator.  Build the library with
``__graft_entry__.build()`` (or ``python -m paper_1701_03549_gb300.build``).
"""
__all__ = ["fire", "synth", "workloads", "parallel"]
