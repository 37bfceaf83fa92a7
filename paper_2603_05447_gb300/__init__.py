"""GB300-native finite-difference Gross-Pitaevskii step on selectively sampled
shell grids (the data-parallel hot path of "Efficient simulation of
Bose-Einstein condensates in nontrivial topologies").

The compute path is the CUDA library ``libgpeshell.so`` (sm_103a) behind the
C ABI in ``include/gpe.h``; ``gpe`` is its ctypes binding.  Importing this
package loads nothing: call ``_build.build()`` once, then use ``gpe``.
"""
__all__ = ["gpe", "inputs"]
