"""GB300-native cyclic compact banded solver (two-level partition + PCR).

``abi``       ctypes binding of the C-ABI (include/cbs.h), same names.
``solver``    torch-facing Plan wrapper (device pointers and streams only).
``workloads`` seeded synthetic inputs shared with the oracle.
``build``     nvcc build of libcbs.so (sm_103a).
"""
__all__ = ["abi", "solver", "workloads", "build"]
