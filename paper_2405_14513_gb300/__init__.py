"""GB300-native FFT estimator of the redshift-space bispectrum multipoles
B_l^m(k1, mu, t) (Gill & Bharadwaj, arXiv:2405.14513).

The compute path lives in the CUDA library ``libbisp.so`` behind the C ABI of
``include/bisp.h``; ``paper_2405_14513_gb300.api`` is a thin ctypes binding
of it.  Submodules are imported lazily so that ``synth`` can be used without
loading the CUDA library.
"""
__all__ = ["api", "synth"]
