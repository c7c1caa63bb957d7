"""GB300 engine for batched electron repulsion integrals with fused fixed-bitwidth
compression (the data-parallel hot path of arXiv 2303.13632).

The compute path is the CUDA library built from ``csrc/`` (C ABI: include/eri.h);
``api`` exposes the same entry points to Python.  Importing this package does not load
the library; the first API call builds/loads it and raises if that fails.
"""
from . import workloads  # noqa: F401

__all__ = ["api", "workloads", "build"]
