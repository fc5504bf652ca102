"""GB300-native Pointing SelfCal hot path (Bhatnagar & Cornwell 2017).

``_abi``   -- ctypes binding of the CUDA library (include/psc.h)
``build``  -- nvcc build of ``_bin/libpsc.so`` for sm_103a
``inputs`` -- seeded synthetic inputs shaped like the paper's workloads
``session``-- device-resident setup of a workload (grid, contexts, data)
"""
