"""GB300-native checkerboard Metropolis sweeps of Ising-type lattices.

The compute path is the CUDA library ``libspn.so`` (``csrc/``) behind the C ABI
declared in ``include/spn.h``; ``spn`` is its thin Python binding.  Importing
this package does not load the library; ``spn.load()`` does, and fails loudly
when the library has not been built.
"""

__all__ = ["inputs", "spn"]
