"""GB300-native Fast Coherent Point Drift EM loop (arXiv 2006.06281).

The compute path is the C-ABI library ``libfcpd.so`` (hand-written sm_103a
CUDA); ``paper_2006_06281_gb300.cpd`` is its thin ctypes binding.  Importing
this package does not load the library; the first call into ``cpd`` does, and
raises if it is missing (there is no CPU fallback).
"""
__all__ = ["cpd", "datagen"]
