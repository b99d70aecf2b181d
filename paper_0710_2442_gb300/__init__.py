"""Wilson-Dirac hopping term, its even-odd form and CG solves on GB300.

The compute path is the C-ABI library ``libwilson_gb300.so`` built from
``csrc/`` (CUDA for sm_103a); ``paper_0710_2442_gb300.wilson`` is its thin
ctypes binding.  Importing this package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["inputs", "model"]
