"""GB300-native HiCR communication path: memcpy between memory slots with
fence and message counters, SPSC/MPSC channels, batching and serving, as a
C-ABI CUDA library (libhicr_gb300.so, declared in include/hicr*.h) plus a
ctypes binding with the same call names.

    from paper_2509_01425_gb300 import build; build.build()
    from paper_2509_01425_gb300 import hicr
"""
__all__ = ["build", "hicr"]
