"""GB300-native Dynamic Ray Tracing (DRT) hot path.

Extrapolates the multipath of one ray-tracing run at t0 over a time lapse (interaction points, delay,
angles, Doppler, validity, complex field) and synthesises H(t, f) with hand-written sm_103a CUDA
kernels behind the C ABI of include/drt.h.  ``drt`` is the ctypes binding, ``inputs`` the seeded
synthetic workloads, ``build`` the nvcc build of the library.
"""
__all__ = ["drt", "inputs", "build"]
