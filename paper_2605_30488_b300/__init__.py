"""B300-native (sm_103a) unified multi-agent Sim(3) Gauss-Newton graph refinement.

The computation lives in libcomo3r.so (hand-written CUDA kernels behind the C ABI of
include/como3r.h); `paper_2605_30488_b300.como3r` is its thin ctypes binding.
"""
__all__ = ["como3r", "build"]
