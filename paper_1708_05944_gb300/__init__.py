"""GB300-native vielbein finite-difference lattice Boltzmann (TVD-RK3 stage hot path).

The solver lives in the C-ABI library ``libvlb.so`` (CUDA kernels for sm_103a);
``paper_1708_05944_gb300.vlb`` is a thin ctypes binding with the same names.
"""
