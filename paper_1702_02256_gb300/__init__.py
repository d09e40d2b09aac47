"""GB300 (sm_103a) Summed Parallel IIR filtering (arXiv:1702.02256).

The compute path is libspiir.so (csrc/, C ABI in include/spiir.h); `spiir`
is its ctypes binding and `inputs` the seeded synthetic workload generator.
"""
