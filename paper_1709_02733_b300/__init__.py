"""B300-native elastic-wave forward/adjoint operator pair (H, H^T) for
transcranial photoacoustic tomography.

The compute path is the C-ABI library ``libpact.so`` (hand-written sm_103a CUDA
kernels); ``pact`` is its thin ctypes binding.  Submodules are imported lazily
so that importing the package does not load the CUDA library.
"""
__all__ = ["pact", "synth", "autograd", "serving"]
