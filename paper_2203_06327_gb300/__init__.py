"""GB300-native two-level BPJD eigensolver (Liang, Wang, Xu): Python face of libbpjd.so.

The CUDA library (``csrc/``, C ABI in ``include/bpjd.h``) holds every step of
the method; this package only builds it (``build``) and marshals arguments
(``binding``).  Importing ``binding`` without a built library raises.
"""

__all__ = ["build", "binding"]
