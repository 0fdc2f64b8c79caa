"""GB300-native block orthogonalization (TreeTSPQR on a locally orthogonal
basis, Dreier & Engwer, arXiv 2204.13393).

The compute path is the CUDA library ``liblo.so`` (C ABI in include/lo.h);
``paper_2204_13393_gb300.lo`` is its thin Python binding.  Importing this
package loads nothing; ``lo`` loads the library on first use and raises if it
has not been built.
"""

__all__ = ["lo", "inputs", "build"]
