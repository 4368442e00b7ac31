"""B300-native coupling-aware Vanka (CAV) multigrid for the implicit immersed-boundary equations.

The compute path is the CUDA library `libcavib.so` (sources in `csrc/`, C ABI in
`include/ib_cav.h`); `api` is a thin ctypes binding with the same call names.  Importing
`api` loads the library and fails loudly if it has not been built -- there is no other
implementation behind it.
"""
__all__ = ["api", "build"]
