"""GB300-native batched satisfiability check for out-of-bounds queries.

The package exposes the C ABI of libscuba (include/scuba.h) through a thin
ctypes binding (``binding``) and a torch-based convenience layer (``api``)
that keeps device buffers in torch tensors. Import of either submodule
fails loudly when the library has not been built.
"""
__all__ = ["binding", "api"]
