"""GB300-native single-level comoving gas advance (Nyx, Almgren et al. 2013).

The compute path is the CUDA library ``libnyxhydro.so`` (sm_103a) behind a
C ABI; ``paper_1301_4498_gb300.hydro`` is its thin ctypes binding.  Input
generators live in ``paper_1301_4498_gb300.workloads``.
"""
__all__ = ["hydro", "workloads"]
