"""GB300-native focused-transport particle pusher (Icarus+PARADISE hot path).

The compute path is the CUDA library libfte_gb300.so (C ABI in include/fte.h);
`paper_2404_12164_gb300.api` is its Python binding.  Importing the package does
not load the library; the first API call does, and fails loudly (ImportError)
if it has not been built with `paper_2404_12164_gb300.build`.
"""
__all__ = ["api", "build"]
