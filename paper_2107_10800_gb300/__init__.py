"""GB300-native solver for suspensions of articulated rigid bodies in Stokes
flow: the constrained mixed mobility-resistance solve of each time step.

The compute path is the C-ABI library ``libam.so`` (CUDA, sm_103a); the
``binding`` module wraps it with ctypes.  ``workloads`` holds the seeded
synthetic inputs.  Importing this package loads nothing; the library is
loaded on first use of the binding.
"""
