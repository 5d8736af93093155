"""B300-native sparse-grid explicit MPM step (sm_103a CUDA behind a C-ABI).

The native library ``libmpm_b300.so`` is loaded lazily on first use of
``paper_2605_28525_b300.mpm``; importing the package itself (for example to use
``workloads``) does not touch CUDA.
"""
__all__ = ["workloads", "mpm"]
