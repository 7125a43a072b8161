"""cgks: compact 8th-order gas-kinetic scheme (arXiv 2001.01570) on one GB300.

The compute path is the CUDA library ``libcgks.so`` (sources in ``csrc/``,
C ABI declared in ``include/cgks.h``); :mod:`.cgks` is its thin ctypes
binding.  :mod:`.workloads` builds seeded initial conditions.  Importing the
package does not load the library; :func:`cgks.load` does, and fails loudly
when it has not been built.
"""
__all__ = ["cgks", "workloads"]
