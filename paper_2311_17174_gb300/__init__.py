"""GB300-native batched Analytic-Kludge EMRI log-likelihood.

The compute path is the CUDA library ``libemri.so`` (hand-written sm_103a
kernels behind the C-ABI declared in ``include/emri.h``); ``emri`` is its thin
ctypes binding.  Importing the package loads nothing: ``emri.load()`` (or the
first call) loads the library and fails loudly when it is missing.
"""
__all__ = ["emri", "inputs"]
