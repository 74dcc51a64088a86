"""GB300-native Particles-on-Demand (PonD) time step, arXiv:2302.00310.

The compute path is the CUDA library ``libpond_gb300.so`` behind the C ABI of
``include/pond.h``; ``pond`` is its thin ctypes binding.  Importing this
package does not load the library; ``pond.lib()`` does, and raises if it is
missing (there is no CPU fallback).
"""
__all__ = ["pond", "workloads"]
