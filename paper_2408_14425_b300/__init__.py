"""Radiance-cascade formal solution on B300 (sm_103a): Python binding of librcx.so.

The compute path is the C-ABI library built from ``csrc/`` (hand-written CUDA);
this package only marshals arguments to it.  ``workloads`` holds the seeded
synthetic inputs.  Importing the package does not load the library; the first
call into ``rcx`` does, and fails loudly if it is missing.
"""
__all__ = ["rcx", "workloads"]
