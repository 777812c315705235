"""GB300-native sixth-order finite-difference compressible hydrodynamics.

The compute path is the C-ABI CUDA library ``libgbfd.so`` (sources under
``csrc/``, declared in ``include/gbfd.h``); ``gbfd`` is its thin ctypes
binding.  Importing this package loads nothing: the library is opened on
first use and an ImportError/OSError is raised if it has not been built.
"""
