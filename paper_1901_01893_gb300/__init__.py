"""GB300-native SMS-MUSSELS reconstruction (Mani et al., arXiv 1901.01893).

The compute path is the C-ABI shared library ``libsmsm.so`` built from
``csrc/`` (hand-written sm_103a CUDA kernels); :mod:`.smsm` is its thin ctypes
binding.  Importing this package does not load the library: the binding loads
it on first use and raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["synth"]
