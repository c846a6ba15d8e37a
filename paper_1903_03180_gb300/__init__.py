"""GB300-native SCPL video retargeting (arXiv 1903.03180).

The CUDA library ``libscpl.so`` (built from ``csrc/``) holds every step of the
retargeting path; ``scpl`` is a thin ctypes binding over its C ABI.  Importing
the package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
__all__ = ["scpl", "synth"]
