"""GB300-native explicit leapfrog stepper for the regularised 2D tsunami wave
equation u_tt = d_x(h_eps d_x u) + d_y(h_eps d_y u) (arXiv:2005.11931, Sec. 2, eq. (2.1)).

The compute path is hand-written CUDA for sm_103a behind the C-ABI library
``libtsu.so`` (declared in ``include/tsu.h``); ``paper_2005_11931_gb300.tsu`` is its
thin Python binding.  Importing this package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["tsu", "inputs"]
