"""GB300-native Newton-Krylov BDDC / FETI-DP deluxe solver for the Bidomain step.

The compute path is the CUDA library ``libbidomain.so`` (sources in
``csrc/``, C-ABI in ``include/bidomain.h``); ``binding`` marshals arguments
to it through ctypes.  Importing this package does not load the library:
``binding.load()`` does, and raises if it has not been built.
"""
__all__ = ["binding", "build"]
