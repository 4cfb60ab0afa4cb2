"""WENO-ZA6 finite-difference right-hand side and SSP-RK3 stepping on GB300.

The compute path is the CUDA library ``libweno.so`` (sources in ``csrc/``,
C-ABI in ``include/weno.h``); ``paper_2603_26272_gb300.weno`` is its thin
ctypes binding.  Nothing is imported here, so the input generators in
``paper_2603_26272_gb300.workloads`` work without a built library.
"""
