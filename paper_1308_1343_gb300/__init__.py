"""GB300-native (sm_103a, FP64) stencil / RK4 level library.

The compute path is the C-ABI library ``libsc_level.so`` built from
``csrc/`` (CUDA kernels and host runtime); ``binding`` marshals arguments to
it with ctypes.  Importing this package loads nothing: ``workloads`` (seeded
inputs) works without a GPU, and ``binding.lib()`` loads the library on
first use and raises if it is missing.
"""
__all__ = ["workloads", "binding", "level"]
