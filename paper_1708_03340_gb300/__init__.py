"""GB300-native HSVD truncation of Hierarchical Tucker tensors.

The compute path lives in the CUDA library ``libhtgb.so`` (sources in
``csrc/``, C-ABI declared in ``include/htgb.h``); ``htgb`` is its thin ctypes
binding.  ``inputs`` draws the seeded synthetic workloads.  Importing this
package loads nothing; the library is loaded on first use of ``htgb`` and
raises if it has not been built.
"""
