"""GB300-native massively parallel algorithm (MPA) for the dispersion-managed
WDM NLSE, Eq. (1), with a same-GPU split-step (SS) comparator.

The compute path is the CUDA library ``libmpa.so`` (hand-written sm_103a
kernels behind the C ABI of ``include/mpa.h``); ``paper_1101_0086_gb300.mpa``
is its thin ctypes binding.  ``paper_1101_0086_gb300.workloads`` builds the
seeded synthetic inputs.
"""
__all__ = ["workloads"]
