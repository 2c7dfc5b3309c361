"""GB300 (sm_103a) continuous Fourier series of Manhattan clips (FCFS hot path).

The CUDA library ``libfcfs.so`` (C ABI in include/fcfs.h) does all the work;
``paper_1010_5562_gb300.fcfs`` is its torch binding.  Build it with
``paper_1010_5562_gb300.build.build()``.
"""
