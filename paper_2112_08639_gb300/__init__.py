"""GB300-native SQ3 hot path (real-space density-kernel method for Kohn-Sham
DFT at high temperature, arXiv 2112.08639).

The compute path is the CUDA library ``libsq3.so`` behind the C ABI declared
in ``include/sq3.h``; ``paper_2112_08639_gb300.sq3`` is its thin ctypes
binding.  ``inputs`` generates the seeded synthetic cells.  Importing this
package does not load the library; ``sq3`` does, and fails loudly if the
library has not been built.
"""
__all__ = ["inputs", "sq3"]
